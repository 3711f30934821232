// Device-side building blocks shared by the kernels of the unrolled COSMO
// path: value loads (f32 / bf16 / f64 storage), deterministic warp and block
// reductions in double, and the batch description passed to every kernel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cosmo {

// cone codes, identical to the C ABI
enum : uint8_t { K_ZERO = 0, K_NONNEG = 1, K_BOX = 2, K_SOC = 3, K_PSD = 4 };

// per-instance flag bits, identical to the C ABI
enum : int32_t {
  F_CG_CAP = 1, F_ADJ_CG_CAP = 2, F_EIG_CAP = 4, F_NONFINITE = 8, F_BAD_PARAM = 16, F_TIMEOUT = 32
};

__device__ __forceinline__ float ldv(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ double ldv(const double* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

template <class T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 5.9604644775390625e-08; };
template <> struct Eps<double> { static constexpr double v = 1.1102230246251565e-16; };

template <class T> struct MaxVal;
template <> struct MaxVal<float> { static constexpr float v = 3.4028234663852886e+38f; };
template <> struct MaxVal<double> { static constexpr double v = 1.7976931348623157e+308; };

__device__ __forceinline__ bool finite_(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_(double v) { return isfinite(v); }

// Butterfly warp sum: every lane ends with the same value, in a fixed order.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The butterfly within aligned groups of L lanes (L a power of two <= 32);
// every lane of a group ends with the group's sum.  L = 32 is warp_sum.
template <int L>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (L == 32) return 0xffffffffu;
  else return ((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1));
}
template <int L>
__device__ __forceinline__ double group_sum(double v) {
  const unsigned mask = group_mask<L>();
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Same butterfly in the value's own type.  On this GPU an FP64 warp
// instruction costs about 16 SM cycles (two FP64 lanes per clock per SM), so
// per-row sums of float data stay in float.
__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_allsum(double v) { return warp_sum(v); }

// Block sum of NV doubles, broadcast to every thread; fixed summation order
// (warp butterflies, then a butterfly over the warps' values in warp 0), so
// results are bitwise reproducible run to run.  Only warp 0 combines the
// warps: with every thread re-adding all warp values, the FP64 adds of a
// 1024-thread block cost microseconds on this GPU's narrow FP64 pipe.
// `sm` needs NV * (blockDim.x / 32) doubles; blockDim.x <= 1024.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[q * nw + warp] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const double t = warp_sum(lane < nw ? sm[q * nw + lane] : 0.0);
      __syncwarp();
      if (lane == 0) sm[q * nw] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = sm[q * nw];
  __syncthreads();
}

// The same for per-thread partials held in the value type T: the warp
// butterflies run in T (float adds on the full-rate pipe), only the
// combination of the warps' values is in double.
template <int NV, class T>
__device__ __forceinline__ void block_sum_t(const T (&v)[NV], double (&out)[NV], double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  T w[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) w[q] = warp_allsum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[q * nw + warp] = (double)w[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const double t = warp_sum(lane < nw ? sm[q * nw + lane] : 0.0);
      __syncwarp();
      if (lane == 0) sm[q * nw] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = sm[q * nw];
  __syncthreads();
}

// Batch description (device pointers), passed by value to every kernel.
// T = iterate type, V = stored matrix value type.
template <class T, class V>
struct Prob {
  int32_t ninst;
  int64_t n_total, m_total;
  const int64_t* col_off;   // [ninst+1]
  const int64_t* row_off;   // [ninst+1]
  const int32_t* row_inst;  // [m_total]
  const int32_t* col_inst;  // [n_total]
  const uint8_t* row_kind;  // [m_total] cone type of each row
  const int64_t* A_rp; const int32_t* A_ci; const V* A_v;     // m_total rows
  const int64_t* AT_rp; const int32_t* AT_ci; const V* AT_v;  // n_total rows
  // P keeps the iterate type: a BF16-rounded P = M'M + reg I can lose
  // positive semidefiniteness (rounding error above its smallest eigenvalue)
  const int64_t* P_rp; const int32_t* P_ci; const T* P_v;     // n_total rows or null
  const T* Pdiag;   // [n_total]
  const T* q;       // [n_total]
  const T* b;       // [m_total]
  const T* box_l;   // [m_total] or null
  const T* box_u;
  int32_t nsoc;
  const int64_t* soc_row0; const int32_t* soc_dim;
  int32_t npsd;
  const int64_t* psd_row0;  // first svec row of each PSD block
  const int32_t* psd_p;
  const int64_t* psd_loff;  // offset of the block's eigenvalues in a lambda slot
  const int64_t* psd_uoff;  // offset of the block's eigenvectors in a U slot
  const int32_t* psd_sched; // PSD blocks, largest p first
  int32_t nrect;            // SOC + PSD blocks (rho rectification)
  const int64_t* rect_row0; const int32_t* rect_rows;
  const int32_t* inst_sched;// instances, most work first (CG)
  // instances whose M = P + sigma I + A'D(rho)A is diagonal for every rho (P
  // diagonal and at most one nonzero per row of A): Jacobi-preconditioned CG
  // reaches the exact solution D^-1 rhs in its first step from any start, so
  // the solve is done in the kernel that forms the right-hand side
  const uint8_t* diag_inst; // [ninst]
  int32_t n_cg;             // instances that need the CG kernel
  const int32_t* cg_sched;  // [n_cg], most work first
};

}  // namespace cosmo
