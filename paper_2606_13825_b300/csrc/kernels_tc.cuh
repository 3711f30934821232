// Daleckii-Krein backward of the PSD projection on the 5th-generation tensor
// cores (tcgen05, TF32 operands, FP32 accumulation in tensor memory).
//
// Per block of order p (Eq. psd-cotangent-dk, Sec. 3.2):
//   S_bar = U (Gamma o (U' G U)) U',   G = smat(g),
// evaluated as four products, each one 128 x pn x pn tcgen05.mma tile
// (pn = p rounded up to 16):
//   1  W  = U' G
//   2  G' = (W U) o Gamma        (Gamma applied while reading the accumulator)
//   3  Y  = U G''                 (G' is symmetric up to rounding)
//   4  S_bar = Y U'               (upper triangle written as svec)
// Every product is formed as A_hi B_hi + A_hi B_lo + A_lo B_hi with each FP32
// operand split into two TF32 parts (x = hi + lo, hi = tf32(x),
// lo = tf32(x - hi)): the result carries about FP32 accuracy instead of the
// 10-bit mantissa of one TF32 product.
//
// Operands live in shared memory in the canonical no-swizzle K-major layout:
// core matrices of 8 rows x 16 bytes (4 TF32), K-adjacent core matrices 128 B
// apart (the descriptor's leading byte offset), 8-row groups pn * 32 + 16 B
// apart (stride byte offset; the extra 16 B spreads the epilogue's stores
// over the banks).  The A operand of an M = 128 tile reads 16 row groups;
// rows past pn only feed accumulator rows that are never read, so the A
// buffers may run into the next buffer (the allocation has a tail for the
// last one).  Rows and K columns past p hold zeros wherever they enter a sum.
//
// One thread issues the MMAs and commits them to an mbarrier; every wait on
// it is bounded and a wait that gives up raises the block's timeout flag.
#pragma once

#include "common.cuh"
#include "kernels_psd.cuh"

namespace cosmo {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), the fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ float tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// TMEM allocation / release: one whole warp
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               :: "r"(smem_u32(slot)), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
               :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count) : "memory");
}

// wait for the phase of the given parity; false after max_iter attempts
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int max_iter) {
  uint32_t done = 0;
  for (int i = 0; i < max_iter && !done; ++i) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
  }
  return done != 0;
}

// 8 consecutive 32-bit columns of this thread's TMEM lane (32x32b shape)
__device__ __forceinline__ void ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace tc

constexpr int DK_TC_NT = 256;    // 8 warps: 4 lane quarters x 2 column halves of the accumulator
constexpr int DK_TC_MAXP = 80;   // largest order whose six operand buffers fit one CTA
constexpr int DK_TC_WAIT = 1 << 22;

__host__ __device__ inline int dk_tc_pn(int p) { return (p + 15) / 16 * 16; }
__host__ __device__ inline int dk_tc_sbo(int pn) { return (pn / 4) * 32 + 4; }    // floats per 8-row group
__host__ __device__ inline int dk_tc_buf(int pn) { return (pn / 8) * dk_tc_sbo(pn); }

// dynamic shared memory for blocks up to order p: six operand buffers, the
// tail an A operand of 128 rows reads past the last one, the eigenvalues,
// the mbarrier and the TMEM address slot
__host__ __device__ inline size_t dk_tc_smem(int p) {
  const int pn = dk_tc_pn(p);
  return (size_t)(6 * dk_tc_buf(pn) + (16 - pn / 8) * dk_tc_sbo(pn) + pn) * sizeof(float) + 64;
}

__device__ __forceinline__ int dk_tc_at(int r, int c, int sbo) {
  return (r >> 3) * sbo + (c >> 2) * 32 + (r & 7) * 4 + (c & 3);
}

// Loewner weight of max(x, 0) for FP32 eigenvalues: same-sign pairs need no
// division (1 for two positive, 0 for two non-positive, 1/2 for two exact
// zeros).  A mixed-sign pair l+ > 0 >= l- whose FP32 gap l+ - l- exceeds
// 2 tau is certainly outside the FP64 gap test's tie band, and its divided
// difference l+ / (l+ - l-) has no cancellation, so it is taken in FP32 (an
// FP64 division costs hundreds of cycles per warp on this part); pairs within
// 2 tau take the FP64 gap test and divided difference.
__device__ __forceinline__ float dk_tc_gamma(float lk, float ll, double tau, float tau2) {
  const bool pk = lk > 0.f, pl = ll > 0.f;
  if (pk && pl) return 1.f;
  if (!pk && !pl) return (lk == 0.f && ll == 0.f) ? 0.5f : 0.f;
  const float lp = pk ? lk : ll, gap = pk ? lk - ll : ll - lk;
  if (gap > tau2) return lp / gap;
  return (float)loewner_relu((double)lk, (double)ll, tau);
}

// D (tensor memory) = A_hi B_hi' + A_hi B_lo' + A_lo B_hi' over K = pn; one
// thread issues, every thread waits (bounded).
__device__ __forceinline__ bool dk_tc_gemm(uint32_t taddr, const float* Ah, const float* Al,
                                           const float* Bh, const float* Bl, int pn, uint64_t* mbar,
                                           uint32_t parity) {
  tc::fence_proxy_async();   // this thread's operand stores, visible to the tensor cores
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (threadIdx.x == 0) {
    const uint32_t idesc = tc::idesc_tf32(128, pn);
    const uint32_t sbo = (uint32_t)dk_tc_sbo(pn) * 4u;
    const float* As[3] = {Ah, Ah, Al};
    const float* Bs[3] = {Bh, Bl, Bh};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const uint32_t a0 = tc::smem_u32(As[t]), b0 = tc::smem_u32(Bs[t]);
      for (int ks = 0; ks < pn / 8; ++ks)
        tc::mma_tf32(taddr, tc::desc(a0 + ks * 256u, 128u, sbo), tc::desc(b0 + ks * 256u, 128u, sbo), idesc,
                     (t | ks) ? 1u : 0u);
    }
    tc::commit(mbar);
  }
  // CTA-uniform: the epilogue's tcgen05.ld must run in every thread of a warp
  const bool ok = __syncthreads_and(tc::mbar_wait(mbar, parity, DK_TC_WAIT));
  tc::fence_after();
  return ok;
}

// f(row, col0, v[8]) for 8 consecutive accumulator columns col0.. of a row
// < pn: warp w reads lanes 32 (w % 4) .. + 31 and the column half w / 4
template <class F>
__device__ __forceinline__ void dk_tc_epilogue(uint32_t taddr, int pn, F f) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (w & 3) + lane;
  const int c0 = (w >> 2) * (pn / 2);
  for (int c = c0; c < c0 + pn / 2; c += 8) {
    float v[8];
    tc::ld8(taddr + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)c, v);
    if (row < pn) f(row, c, v);
  }
}

// 8 consecutive values of row r from column c (a multiple of 8) as two
// 16-byte stores per part (each 4 columns are one core-matrix row)
__device__ __forceinline__ void dk_tc_put8(float* hi, float* lo, int r, int c, int sbo, const float (&v)[8]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float4 a, b;
    a.x = tc::tf32(v[4 * h]); a.y = tc::tf32(v[4 * h + 1]); a.z = tc::tf32(v[4 * h + 2]); a.w = tc::tf32(v[4 * h + 3]);
    b.x = tc::tf32(v[4 * h] - a.x); b.y = tc::tf32(v[4 * h + 1] - a.y);
    b.z = tc::tf32(v[4 * h + 2] - a.z); b.w = tc::tf32(v[4 * h + 3] - a.w);
    const int idx = dk_tc_at(r, c + 4 * h, sbo);
    *reinterpret_cast<float4*>(hi + idx) = a;
    *reinterpret_cast<float4*>(lo + idx) = b;
  }
}

// One block: U column-major p x p (eigenvector k at U[k p ..]), lam [p],
// g / out svec.  Returns false when a wait gave up.
__device__ bool dk_tc_block(int p, const float* __restrict__ U, const float* __restrict__ lam,
                            const float* __restrict__ g, float* __restrict__ out, double tau_rel,
                            unsigned char* smraw) {
  const int pn = dk_tc_pn(p), sbo = dk_tc_sbo(pn), nb = dk_tc_buf(pn);
  float* Uth = reinterpret_cast<float*>(smraw);   // U'  (row k, K i)
  float* Utl = Uth + nb;
  float* Urh = Utl + nb;                          // U   (row i, K k)
  float* Url = Urh + nb;
  float* Xh = Url + nb;                           // G, W, G', Y in turn
  float* Xl = Xh + nb;
  float* lamf = Xl + nb + (16 - pn / 8) * sbo;
  uint64_t* mbar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(lamf + pn) + 7) & ~uintptr_t(7));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  __shared__ double s_tau;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t ncols = pn <= 32 ? 32u : (pn <= 64 ? 64u : 128u);
  if (warp == 0) tc::alloc(tslot, ncols);
  if (tid == 0) tc::mbar_init(mbar, 1);
  // Staging.  U (column-major, contiguous) and g (svec, contiguous) are first
  // copied into shared memory with coalesced loads (U into the G buffer, g
  // into the tail past the last operand buffer, which only the unused rows of
  // a 128-row A operand read); the operands are then written in destination
  // order from there: thread f writes the 16-byte core-matrix row (r,
  // c..c+3), consecutive threads consecutive rows of a core matrix.
  const int q4 = pn / 4;
  const int ps = (p * (p | 1) <= nb) ? (p | 1) : p;   // raw U stride (odd where it fits)
  float* const Ur = Xh;                              // raw U: column k at Ur + k ps
  float* const gr = Xl + nb;                         // raw svec g
  {
    const int d = p * (p + 1) / 2;
#pragma unroll 4
    for (int e = tid; e < p * p; e += DK_TC_NT) {
      const int k = e / p, i = e - k * p;
      Ur[k * ps + i] = U[e];
    }
#pragma unroll 4
    for (int e = tid; e < d; e += DK_TC_NT) gr[e] = g[e];
  }
  __syncthreads();
  for (int f = tid; f < pn * q4; f += DK_TC_NT) {
    const int r = ((f >> 3) / q4) * 8 + (f & 7), c = ((f >> 3) % q4) * 4;
    float ut[4], ur[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = c + j;
      const bool in = r < p && cc < p;
      ut[j] = in ? Ur[r * ps + cc] : 0.f;        // U'(r, cc) = U(cc, r)
      ur[j] = in ? Ur[cc * ps + r] : 0.f;        // U(r, cc)
    }
    const int idx = dk_tc_at(r, c, sbo);
    float4 h, l;
    h = make_float4(tc::tf32(ut[0]), tc::tf32(ut[1]), tc::tf32(ut[2]), tc::tf32(ut[3]));
    l = make_float4(tc::tf32(ut[0] - h.x), tc::tf32(ut[1] - h.y), tc::tf32(ut[2] - h.z), tc::tf32(ut[3] - h.w));
    *reinterpret_cast<float4*>(Uth + idx) = h;
    *reinterpret_cast<float4*>(Utl + idx) = l;
    h = make_float4(tc::tf32(ur[0]), tc::tf32(ur[1]), tc::tf32(ur[2]), tc::tf32(ur[3]));
    l = make_float4(tc::tf32(ur[0] - h.x), tc::tf32(ur[1] - h.y), tc::tf32(ur[2] - h.z), tc::tf32(ur[3] - h.w));
    *reinterpret_cast<float4*>(Urh + idx) = h;
    *reinterpret_cast<float4*>(Url + idx) = l;
  }
  __syncthreads();   // raw U is read: its buffer takes G
  for (int f = tid; f < pn * q4; f += DK_TC_NT) {
    const int r = ((f >> 3) / q4) * 8 + (f & 7), c = ((f >> 3) % q4) * 4;
    float gv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = c + j;
      float g0 = 0.f;
      if (r < p && cc < p) {
        const int i = min(r, cc), jj = max(r, cc);
        g0 = gr[jj * (jj + 1) / 2 + i];
        if (i != jj) g0 *= (float)kInvSqrt2;
      }
      gv[j] = g0;                                // G (symmetric)
    }
    const int idx = dk_tc_at(r, c, sbo);
    const float4 h = make_float4(tc::tf32(gv[0]), tc::tf32(gv[1]), tc::tf32(gv[2]), tc::tf32(gv[3]));
    const float4 l = make_float4(tc::tf32(gv[0] - h.x), tc::tf32(gv[1] - h.y), tc::tf32(gv[2] - h.z),
                                 tc::tf32(gv[3] - h.w));
    *reinterpret_cast<float4*>(Xh + idx) = h;
    *reinterpret_cast<float4*>(Xl + idx) = l;
  }
  for (int k = tid; k < p; k += DK_TC_NT) lamf[k] = lam[k];
  __syncthreads();
  if (warp == 0) {
    float m = 0.f;   // max |lambda| (exact in FP32)
    for (int k = tid; k < p; k += 32) m = fmaxf(m, fabsf(lamf[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (tid == 0) s_tau = tau_rel * fmax(1.0, (double)m);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *tslot;
  const double tau = s_tau;
  const float tau2 = (float)(2.0 * tau);

  // 1: W = U' G  (A = U', B rows j = G(., j))
  bool ok = dk_tc_gemm(taddr, Uth, Utl, Xh, Xl, pn, mbar, 0);
  if (ok) dk_tc_epilogue(taddr, pn, [&](int k, int c, float (&v)[8]) { dk_tc_put8(Xh, Xl, k, c, sbo, v); });
  // 2: G' = (W U) o Gamma  (A = W, B rows l = U(., l)).  G' is symmetric up to
  // rounding; it is stored as it comes (row k, K l), so step 3 forms U G''.
  ok = ok && dk_tc_gemm(taddr, Xh, Xl, Uth, Utl, pn, mbar, 1);
  if (ok)
    dk_tc_epilogue(taddr, pn, [&](int k, int c, float (&v)[8]) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int l = c + j;
        v[j] = (k < p && l < p) ? v[j] * dk_tc_gamma(lamf[k], lamf[l], tau, tau2) : 0.f;
      }
      dk_tc_put8(Xh, Xl, k, c, sbo, v);
    });
  // 3: Y = U G''  (A = U, B rows k = G'(k, .))
  ok = ok && dk_tc_gemm(taddr, Urh, Url, Xh, Xl, pn, mbar, 0);
  if (ok) dk_tc_epilogue(taddr, pn, [&](int i, int c, float (&v)[8]) { dk_tc_put8(Xh, Xl, i, c, sbo, v); });
  // 4: S_bar = Y U'  (A = Y, B rows j = U(j, .)); upper triangle to svec
  ok = ok && dk_tc_gemm(taddr, Xh, Xl, Urh, Url, pn, mbar, 1);
  if (ok)
    dk_tc_epilogue(taddr, pn, [&](int i, int c, float (&v)[8]) {
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = c + jj;
        if (i <= j && j < p) out[j * (j + 1) / 2 + i] = i == j ? v[jj] : v[jj] * (float)kSqrt2;
      }
    });
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(taddr, ncols);
  return ok;
}

// b3 (PSD) on the tensor cores, one CTA per block of order <= DK_TC_MAXP
template <class V>
__global__ void __launch_bounds__(DK_TC_NT) k_psd_bwd_tc(Prob<float, V> P, PsdBwdIO<float> io,
                                                         const float* lam_slot, const float* U_slot,
                                                         double dk_tau_rel, int sched_off, int32_t* flags) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int blk = P.psd_sched[sched_off + blockIdx.x];
  const int64_t row0 = P.psd_row0[blk];
  const bool ok = dk_tc_block(P.psd_p[blk], U_slot + P.psd_uoff[blk], lam_slot + P.psd_loff[blk], io.g + row0,
                              io.vbar + row0, dk_tau_rel, smraw);
  if (!ok && threadIdx.x == 0) atomicOr(&flags[io.row_inst[row0]], F_TIMEOUT);
}

// standalone DK on the tensor cores (blocks laid out as PsdBatch says)
__global__ void __launch_bounds__(DK_TC_NT) k_psd_dk_batch_tc(PsdBatch<float> B, const float* lam_in,
                                                              const float* U_in, const float* g, float* out,
                                                              double dk_tau_rel, int32_t* err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int blk = blockIdx.x;
  const int64_t o = B.off[blk];
  const bool ok = dk_tc_block(B.p[blk], U_in + B.uoff[blk], lam_in + B.loff[blk], g + o, out + o, dk_tau_rel,
                              smraw);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace cosmo
