// Weight-gradient sums of the warm-start and policy MLPs on the tensor cores
// (FP32 batches): part[c][a * KB + b] = sum over the elements n of chunk c
// of A'[a][n] B[b][n], A' = [A; 1] (ka = KA + 1 <= 80 rows), B [KB][N]
// (KB <= 64), i.e. one split-K product D = A' B' per chunk with K = the
// chunk's elements.  Each 32-element K tile is staged in shared memory in
// the no-swizzle K-major core-matrix layout (8 rows x 4 floats per core
// matrix, K-adjacent core matrices 128 B apart, 8-row groups 1040 B apart),
// each FP32 value split into two TF32 parts (x = hi + lo), and one thread
// issues D += A_hi B_hi' + A_hi B_lo' + A_lo B_hi' (tcgen05.mma kind::tf32,
// M = 128, N = 16 / 32 / 64, K = 8 per instruction) into an FP32
// accumulator in tensor memory; the chunk's D is read back with
// tcgen05.ld.  The next tile's global loads are issued into registers while
// the current tile's MMAs run.  A fixed instruction sequence: the sums are
// reproducible.
#pragma once

#include "common.cuh"
#include "kernels_tc.cuh"

namespace cosmo {

constexpr int WSTC_KT = 32;                          // elements per staged K tile
// K-adjacent core matrices 36 floats (144 B) apart instead of 32: a warp's
// staging stores (one row, 32 consecutive elements = 8 core matrices) then
// fall on 32 different banks instead of 8-way on four
constexpr int WSTC_LBO = 36;                         // floats between K-adjacent core matrices
constexpr int WSTC_SBO = (WSTC_KT / 4) * WSTC_LBO + 4;   // floats per 8-row group (1168 B)
constexpr int WSTC_GA = 10;                          // row groups staged for A' (80 rows)
constexpr int WSTC_TAIL = 16 - WSTC_GA;              // an M = 128 A operand reads 16 groups
constexpr int WSTC_WAIT = 1 << 22;

// dynamic shared memory of k_ws_atb_tc<N>: Ah, Al (10 groups each), Bh, Bl
// (N / 8 groups each), the tail the A_lo operand reads past, the mbarrier
// and the tensor-memory address slot
__host__ __device__ inline size_t ws_tc_smem(int N) {
  return (size_t)((2 * WSTC_GA + 2 * (N / 8) + WSTC_TAIL) * WSTC_SBO) * sizeof(float) + 32;
}

__device__ __forceinline__ int ws_tc_at(int r, int c) {
  return (r >> 3) * WSTC_SBO + (c >> 2) * WSTC_LBO + (r & 7) * 4 + (c & 3);
}

template <int N>
__global__ void __launch_bounds__(256) k_ws_atb_tc(int64_t Ntot, int64_t chunk, const float* __restrict__ A,
                                                   int64_t lda, int KA, int ones, const float* __restrict__ B,
                                                   int64_t ldb, int KB, double* __restrict__ part,
                                                   int32_t* __restrict__ err) {
  static_assert(N == 16 || N == 32 || N == 64, "accumulator columns");
  extern __shared__ __align__(16) float tcs[];
  float* Ah = tcs;
  float* Al = Ah + WSTC_GA * WSTC_SBO;
  float* Bh = Al + WSTC_GA * WSTC_SBO;
  float* Bl = Bh + (N / 8) * WSTC_SBO;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bl + (N / 8 + WSTC_TAIL) * WSTC_SBO);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t ncols = N < 32 ? 32u : (uint32_t)N;
  if (warp == 0) tc::alloc(tslot, ncols);
  if (tid == 0) tc::mbar_init(mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *tslot;
  const int ka = KA + ones;
  const int64_t n0 = (int64_t)blockIdx.x * chunk, n1 = min(Ntot, n0 + chunk);
  // Software pipeline: each thread holds the next K tile's values in
  // registers (A': f = tid + 256 u over the 80 x 32 rows x elements; B: over
  // N x 32), loaded while the current tile's MMAs run.
  constexpr int NA = WSTC_GA * 8 * WSTC_KT / 256, NB = N * WSTC_KT / 256;
  float ra[NA], rb[NB];
  auto load_tile = [&](int64_t t0) {
    const int tl = (int)min((int64_t)WSTC_KT, n1 - t0);
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int f = tid + 256 * u, a = f / WSTC_KT, t = f % WSTC_KT;
      ra[u] = (a < ka && t < tl) ? (a < KA ? A[a * lda + t0 + t] : 1.f) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int f = tid + 256 * u, b = f / WSTC_KT, t = f % WSTC_KT;
      rb[u] = (b < KB && t < tl) ? B[b * ldb + t0 + t] : 0.f;
    }
  };
  uint32_t parity = 0;
  bool ok = true, any = false;
  if (n0 < n1) load_tile(n0);
  for (int64_t t0 = n0; t0 < n1 && ok; t0 += WSTC_KT) {
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int f = tid + 256 * u, a = f / WSTC_KT, t = f % WSTC_KT;
      const float hi = tc::tf32(ra[u]);
      const int idx = ws_tc_at(a, t);
      Ah[idx] = hi;
      Al[idx] = tc::tf32(ra[u] - hi);
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int f = tid + 256 * u, b = f / WSTC_KT, t = f % WSTC_KT;
      const float hi = tc::tf32(rb[u]);
      const int idx = ws_tc_at(b, t);
      Bh[idx] = hi;
      Bl[idx] = tc::tf32(rb[u] - hi);
    }
    tc::fence_proxy_async();   // the operand stores, visible to the tensor cores
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      const uint32_t idesc = tc::idesc_tf32(128, N), sbo = WSTC_SBO * 4u, lbo = WSTC_LBO * 4u;
      const float* As[3] = {Ah, Ah, Al};
      const float* Bs[3] = {Bh, Bl, Bh};
#pragma unroll
      for (int pr = 0; pr < 3; ++pr) {
        const uint32_t a0 = tc::smem_u32(As[pr]), b0 = tc::smem_u32(Bs[pr]);
#pragma unroll
        for (int ks = 0; ks < WSTC_KT / 8; ++ks)
          tc::mma_tf32(taddr, tc::desc(a0 + ks * 2u * lbo, lbo, sbo), tc::desc(b0 + ks * 2u * lbo, lbo, sbo), idesc,
                       (any || pr || ks) ? 1u : 0u);
      }
      tc::commit(mbar);
    }
    if (t0 + WSTC_KT < n1) load_tile(t0 + WSTC_KT);   // in flight during the MMAs
    // CTA-uniform (the epilogue's tcgen05.ld runs in every thread of a warp);
    // the wait also frees the operand buffers for the next tile
    ok = __syncthreads_and(tc::mbar_wait(mbar, parity, WSTC_WAIT));
    tc::fence_after();
    parity ^= 1;
    any = true;
  }
  const int npair = ka * KB;
  double* out = part + (int64_t)blockIdx.x * npair;
  if (any && ok) {
    // warp w reads lanes 32 (w % 4) .. + 31 (rows a) and columns [h N/2, (h + 1) N/2), h = w / 4
    const int q = warp & 3, row = 32 * q + lane, c0 = (warp >> 2) * (N / 2);
#pragma unroll
    for (int c = c0; c < c0 + N / 2; c += 8) {
      float v[8];
      tc::ld8(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (row < ka && c + j < KB) out[row * KB + c + j] = (double)v[j];
    }
  } else {
    for (int k = tid; k < npair; k += 256) out[k] = 0.0;
    if (!ok && tid == 0) atomicOr(err, F_TIMEOUT);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(taddr, ncols);
}

}  // namespace cosmo
