// Sparse and elementwise kernels of the unrolled COSMO iteration
// (Sec. 2.2-2.3) and of its reverse pass.
//
// Layout: instances are concatenated; x-like vectors have n_total entries,
// s/y-like vectors m_total.  A is CSR over rows, A' is a second CSR (rows =
// variables) so that every product is a gather (coalesced over rows, no
// atomics, bitwise reproducible).  Per-row loops use one thread per row:
// the rows of the paper's problem classes hold few nonzeros.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace cosmo {

// ---------------------------------------------------------------------------
// a1: rho preparation (App. E rectification), parameter checks, and the
//     Jacobi preconditioner d = diag(P) + sigma + (A o A)' rho (App. D)
// ---------------------------------------------------------------------------
template <class T, class V>
__global__ void k_rho_copy_check(Prob<T, V> P, int32_t K, const T* __restrict__ rho_in,
                                 T* __restrict__ rho_rect, int32_t* flags) {
  const int64_t tot = (int64_t)K * P.m_total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    T v = rho_in[e];
    if (!(v > T(0)) || !finite_(v)) {
      atomicOr(&flags[P.row_inst[e % P.m_total]], F_BAD_PARAM);
    }
    rho_rect[e] = v;
  }
}

// L lanes per (step, SOC/PSD block) -- a warp, or 8 lanes when every block
// has at most 64 rows: replace the rows by their mean
template <class T, class V, int L>
__global__ void k_rho_rectify(Prob<T, V> P, int32_t K, const T* __restrict__ rho_in,
                              T* __restrict__ rho_rect) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / L;
  const int lane = threadIdx.x % L;
  if (w >= (int64_t)K * P.nrect) return;   // whole lane groups
  const int32_t k = (int32_t)(w / P.nrect), c = (int32_t)(w % P.nrect);
  const int64_t r0 = P.rect_row0[c];
  const int32_t nr = P.rect_rows[c];
  const T* src = rho_in + (int64_t)k * P.m_total + r0;
  double acc = 0.0;
  for (int32_t i = lane; i < nr; i += L) acc += (double)src[i];
  acc = group_sum<L>(acc);
  const T mean = (T)(acc / (double)nr);
  T* dst = rho_rect + (int64_t)k * P.m_total + r0;
  for (int32_t i = lane; i < nr; i += L) dst[i] = mean;
}

template <class T, class V>
__global__ void k_alpha_check(Prob<T, V> P, int32_t K, const T* __restrict__ alpha,
                              int32_t* flags) {
  const int64_t tot = (int64_t)K * P.ninst;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    T a = alpha[e];
    if (!(a > T(0) && a < T(2))) atomicOr(&flags[e % P.ninst], F_BAD_PARAM);
  }
}

// dinv[k][j] = 1 / (P_jj + sigma_k + sum_r A_rj^2 rho_k[r])
template <class T, class V>
__global__ void k_precond(Prob<T, V> P, int32_t K, const double* __restrict__ sigma,
                          const T* __restrict__ rho_rect, T* __restrict__ dinv) {
  const int64_t tot = (int64_t)K * P.n_total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = (int32_t)(e / P.n_total);
    const int64_t j = e % P.n_total;
    const T* rho = rho_rect + (int64_t)k * P.m_total;
    T acc = P.Pdiag[j] + (T)sigma[k];
    for (int64_t q = P.AT_rp[j]; q < P.AT_rp[j + 1]; ++q) {
      T a = (T)ldv(P.AT_v, q);
      acc += a * a * rho[P.AT_ci[q]];
    }
    dinv[e] = T(1) / acc;
  }
}

// ---------------------------------------------------------------------------
// a3: xi = sigma x - q + A'(y + rho o (b - s))      (Sec. 2.3, Eq. reduced)
// ---------------------------------------------------------------------------
// For instances with diagonal M the solve x~ = D^-1 xi is done here (dinv is
// the inverse diagonal of M) and written to xt.
template <class T, class V>
__global__ void k_rhs(Prob<T, V> P, double sigma, const T* __restrict__ x,
                      const T* __restrict__ s, const T* __restrict__ y,
                      const T* __restrict__ rho, T* __restrict__ xi,
                      const T* __restrict__ dinv, T* __restrict__ xt) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.n_total;
       j += (int64_t)gridDim.x * blockDim.x) {
    T acc = (T)sigma * x[j] - P.q[j];
    for (int64_t e = P.AT_rp[j]; e < P.AT_rp[j + 1]; ++e) {
      const int32_t r = P.AT_ci[e];
      acc += (T)ldv(P.AT_v, e) * (y[r] + rho[r] * (P.b[r] - s[r]));
    }
    if (P.diag_inst[P.col_inst[j]]) xt[j] = acc * dinv[j];
    else xi[j] = acc;
  }
}

// ---------------------------------------------------------------------------
// a4 / b5: Jacobi-preconditioned CG on M = P + sigma I + A'D(rho)A, one CTA
// per instance, persistent over the CG iterations (no host round trip, no
// inter-CTA waits).  Inner products and the stopping test are in double.
// Stops when ||r||_2 <= tol ||rhs||_2 (recursively updated residual) or at
// maxit (flag bit).  x holds the warm start on entry unless zero_start.
// ---------------------------------------------------------------------------
template <class T>
struct CgArgs {
  const T* rhs;      // [n_total]
  T* x;              // [n_total] out: solution
  const T* x0;       // [n_total] warm start copied into x first (null: x holds it)
  const T* rho;      // [m_total] rectified
  const T* dinv;     // [n_total]
  double sigma;
  T* r; T* p; T* u;  // [n_total] workspace
  T* t;              // [m_total] workspace
  double tol;
  int32_t maxit;
  int32_t zero_start;
  int32_t flag_bit;
  int32_t* flags;
  int32_t* iters;    // [ninst] CG iterations used (may be null)
  unsigned long long* stats;  // [2] total iterations, solves (may be null)
};

// out[row] = f(row, sum_e val[e] x[ci[e]]) for rows [r0, r1) of a CSR matrix,
// CTA-wide, one thread per row, two rows per thread in flight.  Each row is
// read in chunks of 8 entries: the column indices and values of a chunk of
// both rows are loaded first, then all their gathers, so a short row costs
// two dependent round trips instead of two per entry.  The sum runs along the
// row in entry order.
template <bool COH, class T, class V, class F>
__device__ __forceinline__ void cta_csr_rows_c(const int64_t* __restrict__ rp,
                                               const int32_t* __restrict__ ci,
                                               const V* __restrict__ val, const T* __restrict__ x,
                                               int64_t r0, int64_t r1, F f) {
  constexpr int U = 8;
  const int64_t step = blockDim.x;
  for (int64_t rb = r0 + threadIdx.x; rb < r1; rb += 2 * step) {
    int64_t e[2], eend[2];
    T acc[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t r = rb + u * step;
      const bool ok = r < r1;
      e[u] = ok ? rp[r] : 0;
      eend[u] = ok ? rp[r + 1] : 0;
      acc[u] = T(0);
    }
    while (e[0] < eend[0] || e[1] < eend[1]) {
      int32_t c[2][U];
      T v[2][U];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t idx = e[u] + k;
          const bool ok = idx < eend[u];
          c[u][k] = ok ? ci[idx] : -1;
          v[u][k] = ok ? (T)ldv(val, idx) : T(0);
        }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int k = 0; k < U; ++k)
          if (c[u][k] >= 0) acc[u] += v[u][k] * (COH ? __ldcg(x + c[u][k]) : x[c[u][k]]);
#pragma unroll
      for (int u = 0; u < 2; ++u) e[u] = min(e[u] + U, eend[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t r = rb + u * step;
      if (r < r1) f(r, acc[u]);
    }
  }
}

template <class T, class V, class F>
__device__ __forceinline__ void cta_csr_rows(const int64_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci,
                                             const V* __restrict__ val, const T* __restrict__ x,
                                             int64_t r0, int64_t r1, F f) {
  cta_csr_rows_c<false>(rp, ci, val, x, r0, r1, f);
}

// CTA barrier (CS = 1) or cluster barrier over the CS CTAs of an instance
template <int CS>
__device__ __forceinline__ void cg_sync() {
  if constexpr (CS == 1) __syncthreads();
  else cooperative_groups::this_cluster().sync();
}

// Sum of NV doubles over the CTAs of a cluster (every thread holds its CTA's
// total on entry): each CTA publishes its totals in shared memory, then every
// CTA reads all of them through distributed shared memory in rank order, so
// all CTAs hold the same bitwise result.  Two slot sets alternate, so one
// cluster barrier per reduction suffices (a slot set is rewritten only after
// the next reduction's barrier, which every reader of it has passed).
template <int CS, int NV>
__device__ __forceinline__ void cg_cluster_sum(double (&v)[NV], double* slots, int& par) {
  if constexpr (CS > 1) {
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    double* my = slots + par * NV;
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) my[q] = v[q];
    }
    cl.sync();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = 0.0;
    for (int rk = 0; rk < CS; ++rk) {
      const double* ps = cl.map_shared_rank(my, rk);
#pragma unroll
      for (int q = 0; q < NV; ++q) v[q] += ps[q];
    }
    par ^= 1;
  }
}

// u = M v on this CTA's columns [c0, c1) of one instance (its rows [r0, r1)
// produce t); with CS > 1 the CTAs of a cluster split the instance's rows and
// columns and v, t are gathered through L2.
template <int CS, class T, class V>
__device__ __forceinline__ void cta_matvec_cl(const Prob<T, V>& P, const CgArgs<T>& a,
                                              const T* __restrict__ v, T* __restrict__ u,
                                              int64_t c0, int64_t c1, int64_t r0, int64_t r1) {
  constexpr bool COH = CS > 1;
  T* __restrict__ t = a.t;
  const T* __restrict__ rho = a.rho;
  cta_csr_rows_c<COH, T, V>(P.A_rp, P.A_ci, P.A_v, v, r0, r1,
                            [&](int64_t r, T acc) { t[r] = rho[r] * acc; });
  cg_sync<CS>();
  const T sig = (T)a.sigma;
  if (P.P_rp) {
    // u = sigma v + P v, then u += A' t
    cta_csr_rows_c<COH, T, T>(P.P_rp, P.P_ci, P.P_v, v, c0, c1,
                              [&](int64_t j, T acc) { u[j] = sig * v[j] + acc; });
    cta_csr_rows_c<COH, T, V>(P.AT_rp, P.AT_ci, P.AT_v, (const T*)t, c0, c1,
                              [&](int64_t j, T acc) { u[j] += acc; });
  } else {
    cta_csr_rows_c<COH, T, V>(P.AT_rp, P.AT_ci, P.AT_v, (const T*)t, c0, c1,
                              [&](int64_t j, T acc) { u[j] = sig * v[j] + acc; });
  }
  __syncthreads();
}

template <class T, class V>
__device__ __forceinline__ void cta_matvec(const Prob<T, V>& P, const CgArgs<T>& a,
                                           const T* __restrict__ v, T* __restrict__ u,
                                           int64_t c0, int64_t c1, int64_t r0, int64_t r1) {
  cta_matvec_cl<1>(P, a, v, u, c0, c1, r0, r1);
}

// a4 / b5: Jacobi-PCG on one instance per CTA (CS = 1) or per cluster of CS
// CTAs (launched with that cluster size), each CTA owning a contiguous slice
// of the instance's rows and columns.  Stop when ||r||^2 <= tol^2 ||rhs||^2
// (recursively updated r) or at the cap; dots in double.
template <class T, class V, int NT, int CS = 1>
__global__ void __launch_bounds__(NT) k_pcg(Prob<T, V> P, CgArgs<T> a) {
  __shared__ double sm[3 * (NT / 32)];
  __shared__ double slots[2 * 3];
  int par = 0;
  int cid = blockIdx.x, rank = 0;
  if constexpr (CS > 1) {
    cid = blockIdx.x / CS;
    rank = (int)cooperative_groups::this_cluster().block_rank();
  }
  const int32_t inst = P.cg_sched ? P.cg_sched[cid] : P.inst_sched[cid];
  const int64_t ic0 = P.col_off[inst], ic1 = P.col_off[inst + 1];
  const int64_t ir0 = P.row_off[inst], ir1 = P.row_off[inst + 1];
  if (ic1 == ic0) return;   // the whole cluster (same instance)
  const int64_t cw = (ic1 - ic0 + CS - 1) / CS, rw = (ir1 - ir0 + CS - 1) / CS;
  const int64_t c0 = ic0 + min(ic1 - ic0, rank * cw), c1 = ic0 + min(ic1 - ic0, (rank + 1) * cw);
  const int64_t r0 = ir0 + min(ir1 - ir0, rank * rw), r1 = ir0 + min(ir1 - ir0, (rank + 1) * rw);
  T* __restrict__ x = a.x;
  T* __restrict__ r = a.r;
  T* __restrict__ p = a.p;
  T* __restrict__ u = a.u;
  if (a.zero_start) {
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) x[j] = T(0);
  } else {
    if (a.x0 && a.x0 != a.x)
      for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) x[j] = a.x0[j];
    cg_sync<CS>();
    cta_matvec_cl<CS>(P, a, x, u, c0, c1, r0, r1);
  }
  double s3[3] = {0.0, 0.0, 0.0};   // rz, rr, bb
  for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
    const T bj = a.rhs[j];
    const T rj = a.zero_start ? bj : bj - u[j];
    const T zj = a.dinv[j] * rj;
    r[j] = rj;
    p[j] = zj;
    s3[0] += (double)rj * (double)zj;
    s3[1] += (double)rj * (double)rj;
    s3[2] += (double)bj * (double)bj;
  }
  block_sum<3>(s3, sm);
  cg_cluster_sum<CS, 3>(s3, slots, par);   // (its barrier, or block_sum's, publishes p)
  double rz = s3[0], rr = s3[1];
  const double thr = a.tol * a.tol * s3[2];
  int32_t it = 0;
  if (s3[2] == 0.0) {
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) x[j] = T(0);
    rr = 0.0;
  }
  while (rr > thr && it < a.maxit) {
    cta_matvec_cl<CS>(P, a, p, u, c0, c1, r0, r1);
    double s1[1] = {0.0};
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) s1[0] += (double)p[j] * (double)u[j];
    block_sum<1>(s1, sm);
    cg_cluster_sum<CS, 1>(s1, slots, par);
    if (!(s1[0] > 0.0)) break;  // breakdown (p = 0 or non-finite): stop, flagged below
    const T al = (T)(rz / s1[0]);
    double s2[2] = {0.0, 0.0};
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
      x[j] += al * p[j];
      const T rj = r[j] - al * u[j];
      r[j] = rj;
      const T zj = a.dinv[j] * rj;
      s2[0] += (double)rj * (double)zj;
      s2[1] += (double)rj * (double)rj;
    }
    block_sum<2>(s2, sm);
    cg_cluster_sum<CS, 2>(s2, slots, par);
    const T be = (T)(s2[0] / rz);
    rz = s2[0];
    rr = s2[1];
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) p[j] = a.dinv[j] * r[j] + be * p[j];
    cg_sync<CS>();
    ++it;
  }
  // no CTA leaves while a peer may still read its slots (after a break, or
  // when the loop did not run)
  if constexpr (CS > 1) cooperative_groups::this_cluster().sync();
  if (rank == 0 && threadIdx.x == 0) {
    if (rr > thr) atomicOr(&a.flags[inst], a.flag_bit);
    if (!(rr == rr)) atomicOr(&a.flags[inst], F_NONFINITE);
    if (a.iters) a.iters[inst] = it;
    if (a.stats) {
      atomicAdd(&a.stats[0], (unsigned long long)it);
      atomicAdd(&a.stats[1], 1ull);
    }
  }
}

// out[row] = f(row, sum_e val[e] x[ci[e]]) for rows [r0, r1), one warp,
// lane l taking rows r0 + l, r0 + l + 32, ...: two rows per lane in flight,
// each read in chunks of 8 entries (indices and values, then the gathers);
// the sum runs along the row in entry order.
template <class T, class V, class F>
__device__ __forceinline__ void warp_csr_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                              const V* __restrict__ val, const T* __restrict__ x, int64_t r0,
                                              int64_t r1, int lane, F f) {
  constexpr int U = 8;
  for (int64_t rb = r0 + lane; rb < r1; rb += 64) {
    int64_t e[2], eend[2];
    T acc[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t r = rb + u * 32;
      const bool ok = r < r1;
      e[u] = ok ? rp[r] : 0;
      eend[u] = ok ? rp[r + 1] : 0;
      acc[u] = T(0);
    }
    while (e[0] < eend[0] || e[1] < eend[1]) {
      int32_t c[2][U];
      T v[2][U];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t idx = e[u] + k;
          const bool ok = idx < eend[u];
          c[u][k] = ok ? ci[idx] : -1;
          v[u][k] = ok ? (T)ldv(val, idx) : T(0);
        }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int k = 0; k < U; ++k)
          if (c[u][k] >= 0) acc[u] += v[u][k] * x[c[u][k]];
#pragma unroll
      for (int u = 0; u < 2; ++u) e[u] = min(e[u] + U, eend[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t r = rb + u * 32;
      if (r < r1) f(r, acc[u]);
    }
  }
}

// a4 / b5 for many small instances: the Jacobi-PCG of k_pcg with one WARP per
// instance (WPB warps per CTA, option cg_cluster = -4).  A warp needs no CTA
// barrier or block reduction: its phases are ordered by __syncwarp (which
// also orders the warp's global writes), and the inner products are double
// warp sums by shuffles.  The same iteration, stopping rule, warm start, cap
// and flags as k_pcg; the inner products are summed in another order, so
// iterates agree with k_pcg to rounding, not bit for bit.  Measured on the
// covariance-steering workload (512 instances, n + m ~ 1,850): 20.5 ms of CG
// per step against 12.1 for k_pcg_local -- one warp's chains of gathers
// through L2 hide less latency than a CTA with the instance's matrices staged
// in shared memory -- so it is an option and an autotuner candidate only.
template <class T, class V, int WPB>
__global__ void __launch_bounds__(32 * WPB) k_pcg_warp(Prob<T, V> P, CgArgs<T> a) {
  const int lane = threadIdx.x & 31;
  const int cid = blockIdx.x * WPB + (threadIdx.x >> 5);
  if (cid >= P.n_cg) return;                 // whole warps: no CTA barrier below
  const int32_t inst = P.cg_sched[cid];
  const int64_t c0 = P.col_off[inst], c1 = P.col_off[inst + 1];
  const int64_t r0 = P.row_off[inst], r1 = P.row_off[inst + 1];
  if (c1 == c0) return;
  T* __restrict__ x = a.x;
  T* __restrict__ r = a.r;
  T* __restrict__ p = a.p;
  T* __restrict__ u = a.u;
  T* __restrict__ t = a.t;
  const T* __restrict__ rho = a.rho;
  const T sig = (T)a.sigma;
  // u = M v = sigma v + P v + A' (rho o (A v)) on this instance
  auto matvec = [&](const T* __restrict__ v) {
    warp_csr_rows<T, V>(P.A_rp, P.A_ci, P.A_v, v, r0, r1, lane, [&](int64_t q, T acc) { t[q] = rho[q] * acc; });
    __syncwarp();
    if (P.P_rp) {
      warp_csr_rows<T, T>(P.P_rp, P.P_ci, P.P_v, v, c0, c1, lane, [&](int64_t j, T acc) { u[j] = sig * v[j] + acc; });
      warp_csr_rows<T, V>(P.AT_rp, P.AT_ci, P.AT_v, (const T*)t, c0, c1, lane, [&](int64_t j, T acc) { u[j] += acc; });
    } else {
      warp_csr_rows<T, V>(P.AT_rp, P.AT_ci, P.AT_v, (const T*)t, c0, c1, lane,
                          [&](int64_t j, T acc) { u[j] = sig * v[j] + acc; });
    }
    __syncwarp();
  };
  if (a.zero_start) {
    for (int64_t j = c0 + lane; j < c1; j += 32) x[j] = T(0);
  } else {
    if (a.x0 && a.x0 != a.x)
      for (int64_t j = c0 + lane; j < c1; j += 32) x[j] = a.x0[j];
    __syncwarp();
    matvec(x);
  }
  double rz = 0.0, rr = 0.0, bb = 0.0;
  for (int64_t j = c0 + lane; j < c1; j += 32) {
    const T bj = a.rhs[j];
    const T rj = a.zero_start ? bj : bj - u[j];
    const T zj = a.dinv[j] * rj;
    r[j] = rj;
    p[j] = zj;
    rz += (double)rj * (double)zj;
    rr += (double)rj * (double)rj;
    bb += (double)bj * (double)bj;
  }
  rz = warp_sum(rz);
  rr = warp_sum(rr);
  bb = warp_sum(bb);
  __syncwarp();
  const double thr = a.tol * a.tol * bb;
  int32_t it = 0;
  if (bb == 0.0) {
    for (int64_t j = c0 + lane; j < c1; j += 32) x[j] = T(0);
    rr = 0.0;
  }
  while (rr > thr && it < a.maxit) {
    matvec(p);
    double pu = 0.0;
    for (int64_t j = c0 + lane; j < c1; j += 32) pu += (double)p[j] * (double)u[j];
    pu = warp_sum(pu);
    if (!(pu > 0.0)) break;                  // breakdown: stop, flagged below
    const T al = (T)(rz / pu);
    double s0 = 0.0, s1 = 0.0;
    for (int64_t j = c0 + lane; j < c1; j += 32) {
      x[j] += al * p[j];
      const T rj = r[j] - al * u[j];
      r[j] = rj;
      const T zj = a.dinv[j] * rj;
      s0 += (double)rj * (double)zj;
      s1 += (double)rj * (double)rj;
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    const T be = (T)(s0 / rz);
    rz = s0;
    rr = s1;
    for (int64_t j = c0 + lane; j < c1; j += 32) p[j] = a.dinv[j] * r[j] + be * p[j];
    __syncwarp();
    ++it;
  }
  if (lane == 0) {
    if (rr > thr) atomicOr(&a.flags[inst], a.flag_bit);
    if (!(rr == rr)) atomicOr(&a.flags[inst], F_NONFINITE);
    if (a.iters) a.iters[inst] = it;
    if (a.stats) {
      atomicAdd(&a.stats[0], (unsigned long long)it);
      atomicAdd(&a.stats[1], 1ull);
    }
  }
}

// cta_csr_rows_c with the gathered vector in shared memory: entry c of the
// instance-local vector xl is column (c + base) of the batch
template <class T, class V, class F>
__device__ __forceinline__ void cta_csr_rows_local(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   const V* __restrict__ val, const T* xl, int64_t base, int64_t r0,
                                                   int64_t r1, F f) {
  constexpr int U = 8;
  const int64_t step = blockDim.x;
  for (int64_t rb = r0 + threadIdx.x; rb < r1; rb += 2 * step) {
    int64_t e[2], eend[2];
    T acc[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t r = rb + u * step;
      const bool ok = r < r1;
      e[u] = ok ? rp[r] : 0;
      eend[u] = ok ? rp[r + 1] : 0;
      acc[u] = T(0);
    }
    while (e[0] < eend[0] || e[1] < eend[1]) {
      int32_t c[2][U];
      T v[2][U];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t idx = e[u] + k;
          const bool ok = idx < eend[u];
          c[u][k] = ok ? (int32_t)(ci[idx] - base) : -1;
          v[u][k] = ok ? (T)ldv(val, idx) : T(0);
        }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int k = 0; k < U; ++k)
          if (c[u][k] >= 0) acc[u] += v[u][k] * xl[c[u][k]];
#pragma unroll
      for (int u = 0; u < 2; ++u) e[u] = min(e[u] + U, eend[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t r = rb + u * step;
      if (r < r1) f(r, acc[u]);
    }
  }
}

// k_pcg (one CTA per instance) with the instance's vectors x, r, p, u, the
// Jacobi diagonal and t = rho o (A v) in shared memory: the matrix streams
// from L2 / HBM while every gather and update stays on chip.  The same
// arithmetic in the same order as k_pcg, so the iterates are identical.
// Dynamic shared memory: (5 n_i + m_i) reals for the largest instance.
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_pcg_smem(Prob<T, V> P, CgArgs<T> a) {
  __shared__ double sm[3 * (NT / 32)];
  extern __shared__ __align__(16) unsigned char cg_sm[];
  const int32_t inst = P.cg_sched ? P.cg_sched[blockIdx.x] : P.inst_sched[blockIdx.x];
  const int64_t c0 = P.col_off[inst], c1 = P.col_off[inst + 1];
  const int64_t r0 = P.row_off[inst], r1 = P.row_off[inst + 1];
  if (c1 == c0) return;
  const int64_t nl = c1 - c0;
  T* sx = reinterpret_cast<T*>(cg_sm);
  T* sr = sx + nl;
  T* sp = sr + nl;
  T* su = sp + nl;
  T* sd = su + nl;
  T* st = sd + nl;
  const T sig = (T)a.sigma;
  const T* __restrict__ rho = a.rho;
  // u = (P + sigma I + A' D(rho) A) v on the instance, v and u in shared memory
  auto matvec = [&](const T* v, T* u) {
    cta_csr_rows_local<T, V>(P.A_rp, P.A_ci, P.A_v, v, c0, r0, r1,
                             [&](int64_t r, T acc) { st[r - r0] = rho[r] * acc; });
    __syncthreads();
    if (P.P_rp) {
      cta_csr_rows_local<T, T>(P.P_rp, P.P_ci, P.P_v, v, c0, c0, c1,
                               [&](int64_t j, T acc) { u[j - c0] = sig * v[j - c0] + acc; });
      cta_csr_rows_local<T, V>(P.AT_rp, P.AT_ci, P.AT_v, (const T*)st, r0, c0, c1,
                               [&](int64_t j, T acc) { u[j - c0] += acc; });
    } else {
      cta_csr_rows_local<T, V>(P.AT_rp, P.AT_ci, P.AT_v, (const T*)st, r0, c0, c1,
                               [&](int64_t j, T acc) { u[j - c0] = sig * v[j - c0] + acc; });
    }
    __syncthreads();
  };
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) {
    sd[j - c0] = a.dinv[j];
    sx[j - c0] = a.zero_start ? T(0) : (a.x0 ? a.x0[j] : a.x[j]);
  }
  __syncthreads();
  if (!a.zero_start) matvec(sx, su);
  double s3[3] = {0.0, 0.0, 0.0};   // rz, rr, bb
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) {
    const int64_t l = j - c0;
    const T bj = a.rhs[j];
    const T rj = a.zero_start ? bj : bj - su[l];
    const T zj = sd[l] * rj;
    sr[l] = rj;
    sp[l] = zj;
    s3[0] += (double)rj * (double)zj;
    s3[1] += (double)rj * (double)rj;
    s3[2] += (double)bj * (double)bj;
  }
  block_sum<3>(s3, sm);
  double rz = s3[0], rr = s3[1];
  const double thr = a.tol * a.tol * s3[2];
  int32_t it = 0;
  if (s3[2] == 0.0) {
    for (int64_t l = threadIdx.x; l < nl; l += NT) sx[l] = T(0);
    rr = 0.0;
  }
  while (rr > thr && it < a.maxit) {
    matvec(sp, su);
    double s1[1] = {0.0};
    for (int64_t l = threadIdx.x; l < nl; l += NT) s1[0] += (double)sp[l] * (double)su[l];
    block_sum<1>(s1, sm);
    if (!(s1[0] > 0.0)) break;  // breakdown (p = 0 or non-finite): stop, flagged below
    const T al = (T)(rz / s1[0]);
    double s2[2] = {0.0, 0.0};
    for (int64_t l = threadIdx.x; l < nl; l += NT) {
      sx[l] += al * sp[l];
      const T rj = sr[l] - al * su[l];
      sr[l] = rj;
      const T zj = sd[l] * rj;
      s2[0] += (double)rj * (double)zj;
      s2[1] += (double)rj * (double)rj;
    }
    block_sum<2>(s2, sm);
    const T be = (T)(s2[0] / rz);
    rz = s2[0];
    rr = s2[1];
    for (int64_t l = threadIdx.x; l < nl; l += NT) sp[l] = sd[l] * sr[l] + be * sp[l];
    __syncthreads();
    ++it;
  }
  __syncthreads();
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) a.x[j] = sx[j - c0];
  if (threadIdx.x == 0) {
    if (rr > thr) atomicOr(&a.flags[inst], a.flag_bit);
    if (!(rr == rr)) atomicOr(&a.flags[inst], F_NONFINITE);
    if (a.iters) a.iters[inst] = it;
    if (a.stats) {
      atomicAdd(&a.stats[0], (unsigned long long)it);
      atomicAdd(&a.stats[1], 1ull);
    }
  }
}

// A CSR block of one instance staged in shared memory with local indices
template <class V>
struct SmemCsr {
  const int32_t* rp;   // [rows + 1], from 0
  const int32_t* ci;   // local column indices
  const V* v;
};

// bytes of the staged copy of rows [r0, r1) of a batch CSR matrix (each array 16-byte aligned)
__host__ __device__ inline size_t smem_csr_bytes(int64_t rows, int64_t nnz, size_t vsize) {
  auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
  return al(sizeof(int32_t) * (rows + 1)) + al(sizeof(int32_t) * nnz) + al(vsize * nnz);
}

// copy rows [r0, r1) of (rp, ci, val) to shared memory at *cur, columns shifted by -cbase
template <class V>
__device__ inline SmemCsr<V> stage_csr(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                       const V* __restrict__ val, int64_t r0, int64_t r1, int64_t cbase,
                                       unsigned char*& cur) {
  auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const int64_t e0 = rp[r0], nnz = rp[r1] - e0, rows = r1 - r0;
  int32_t* srp = reinterpret_cast<int32_t*>(cur);
  cur += al(sizeof(int32_t) * (rows + 1));
  int32_t* sci = reinterpret_cast<int32_t*>(cur);
  cur += al(sizeof(int32_t) * nnz);
  V* sv = reinterpret_cast<V*>(cur);
  cur += al(sizeof(V) * nnz);
  for (int64_t r = threadIdx.x; r <= rows; r += blockDim.x) srp[r] = (int32_t)(rp[r0 + r] - e0);
  for (int64_t e = threadIdx.x; e < nnz; e += blockDim.x) {
    sci[e] = (int32_t)(ci[e0 + e] - cbase);
    sv[e] = val[e0 + e];
  }
  return SmemCsr<V>{srp, sci, sv};
}

// plain (shared-memory) loads of a staged value: ldv's non-coherent global
// loads must not be used on shared memory
__device__ __forceinline__ float smv(const float* p, int32_t i) { return p[i]; }
__device__ __forceinline__ double smv(const double* p, int32_t i) { return p[i]; }
__device__ __forceinline__ float smv(const __nv_bfloat16* p, int32_t i) { return __bfloat162float(p[i]); }

// out = f(row, sum over the row's entries in order of val * xl[col]), thread per row
template <class T, class V, class F>
__device__ __forceinline__ void smem_csr_rows(const SmemCsr<V>& M, const T* xl, int64_t rows, F f) {
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
    T acc = T(0);
    for (int32_t e = M.rp[r]; e < M.rp[r + 1]; ++e) acc += (T)smv(M.v, e) * xl[M.ci[e]];
    f(r, acc);
  }
}

// k_pcg_smem with the instance's A, A' and P staged in shared memory as
// well: every phase of an iteration stays on chip (small instances, where
// the dependent row-pointer / index / gather loads from L2 bound the
// iteration).  Same sums in the same order per row and per dot product.
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_pcg_local(Prob<T, V> P, CgArgs<T> a) {
  __shared__ double sm[3 * (NT / 32)];
  extern __shared__ __align__(16) unsigned char cg_sm[];
  const int32_t inst = P.cg_sched ? P.cg_sched[blockIdx.x] : P.inst_sched[blockIdx.x];
  const int64_t c0 = P.col_off[inst], c1 = P.col_off[inst + 1];
  const int64_t r0 = P.row_off[inst], r1 = P.row_off[inst + 1];
  if (c1 == c0) return;
  const int64_t nl = c1 - c0, ml = r1 - r0;
  T* sx = reinterpret_cast<T*>(cg_sm);
  T* sr = sx + nl;
  T* sp = sr + nl;
  T* su = sp + nl;
  T* sd = su + nl;
  T* st = sd + nl;
  unsigned char* cur = cg_sm + ((sizeof(T) * (5 * nl + ml) + 15) & ~(size_t)15);
  const SmemCsr<V> mA = stage_csr<V>(P.A_rp, P.A_ci, P.A_v, r0, r1, c0, cur);
  const SmemCsr<V> mAT = stage_csr<V>(P.AT_rp, P.AT_ci, P.AT_v, c0, c1, r0, cur);
  SmemCsr<T> mP{nullptr, nullptr, nullptr};
  if (P.P_rp) mP = stage_csr<T>(P.P_rp, P.P_ci, P.P_v, c0, c1, c0, cur);
  const T sig = (T)a.sigma;
  const T* __restrict__ rho = a.rho;
  auto matvec = [&](const T* v, T* u) {
    smem_csr_rows<T, V>(mA, v, ml, [&](int64_t r, T acc) { st[r] = rho[r0 + r] * acc; });
    __syncthreads();
    if (P.P_rp) {
      smem_csr_rows<T, T>(mP, v, nl, [&](int64_t j, T acc) { u[j] = sig * v[j] + acc; });
      smem_csr_rows<T, V>(mAT, (const T*)st, nl, [&](int64_t j, T acc) { u[j] += acc; });
    } else {
      smem_csr_rows<T, V>(mAT, (const T*)st, nl, [&](int64_t j, T acc) { u[j] = sig * v[j] + acc; });
    }
    __syncthreads();
  };
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) {
    sd[j - c0] = a.dinv[j];
    sx[j - c0] = a.zero_start ? T(0) : (a.x0 ? a.x0[j] : a.x[j]);
  }
  __syncthreads();
  if (!a.zero_start) matvec(sx, su);
  double s3[3] = {0.0, 0.0, 0.0};   // rz, rr, bb
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) {
    const int64_t l = j - c0;
    const T bj = a.rhs[j];
    const T rj = a.zero_start ? bj : bj - su[l];
    const T zj = sd[l] * rj;
    sr[l] = rj;
    sp[l] = zj;
    s3[0] += (double)rj * (double)zj;
    s3[1] += (double)rj * (double)rj;
    s3[2] += (double)bj * (double)bj;
  }
  block_sum<3>(s3, sm);
  double rz = s3[0], rr = s3[1];
  const double thr = a.tol * a.tol * s3[2];
  int32_t it = 0;
  if (s3[2] == 0.0) {
    for (int64_t l = threadIdx.x; l < nl; l += NT) sx[l] = T(0);
    rr = 0.0;
  }
  while (rr > thr && it < a.maxit) {
    matvec(sp, su);
    double s1[1] = {0.0};
    for (int64_t l = threadIdx.x; l < nl; l += NT) s1[0] += (double)sp[l] * (double)su[l];
    block_sum<1>(s1, sm);
    if (!(s1[0] > 0.0)) break;  // breakdown (p = 0 or non-finite): stop, flagged below
    const T al = (T)(rz / s1[0]);
    double s2[2] = {0.0, 0.0};
    for (int64_t l = threadIdx.x; l < nl; l += NT) {
      sx[l] += al * sp[l];
      const T rj = sr[l] - al * su[l];
      sr[l] = rj;
      const T zj = sd[l] * rj;
      s2[0] += (double)rj * (double)zj;
      s2[1] += (double)rj * (double)rj;
    }
    block_sum<2>(s2, sm);
    const T be = (T)(s2[0] / rz);
    rz = s2[0];
    rr = s2[1];
    for (int64_t l = threadIdx.x; l < nl; l += NT) sp[l] = sd[l] * sr[l] + be * sp[l];
    __syncthreads();
    ++it;
  }
  __syncthreads();
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) a.x[j] = sx[j - c0];
  if (threadIdx.x == 0) {
    if (rr > thr) atomicOr(&a.flags[inst], a.flag_bit);
    if (!(rr == rr)) atomicOr(&a.flags[inst], F_NONFINITE);
    if (a.iters) a.iters[inst] = it;
    if (a.stats) {
      atomicAdd(&a.stats[0], (unsigned long long)it);
      atomicAdd(&a.stats[1], 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// a5, a6 (separable cones), a8: s~ = b - A x~, relaxation, projection of
// v = alpha s~ + (1-alpha) s + y/rho on zero / orthant / box rows, dual update;
// x+ = alpha x~ + (1 - alpha) x.  SOC and PSD rows only store s~ here.
// ---------------------------------------------------------------------------
template <class T>
struct StepPtrs {
  const T* x; const T* s; const T* y;   // z^k
  T* xn; T* sn; T* yn;                  // z^{k+1}
  const T* rho;                         // rectified rho^k [m_total]
  const T* alpha;                       // [ninst]
  const T* xt;                          // x~ [n_total]
  T* st;                                // s~ [m_total] (tape)
  T* lam; T* U;                         // PSD eigen tape slot
  int32_t* flags;
};

template <class T, class V>
__global__ void k_post(Prob<T, V> P, StepPtrs<T> q) {
  const int64_t tot = P.m_total + P.n_total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < P.m_total) {
      const int64_t r = e;
      T acc = T(0);
      for (int64_t k = P.A_rp[r]; k < P.A_rp[r + 1]; ++k) acc += (T)ldv(P.A_v, k) * q.xt[P.A_ci[k]];
      const T st = P.b[r] - acc;
      q.st[r] = st;
      const uint8_t kind = P.row_kind[r];
      if (kind <= K_BOX) {
        const T al = q.alpha[P.row_inst[r]];
        const T rh = q.rho[r];
        const T sh = al * st + (T(1) - al) * q.s[r];
        const T v = sh + q.y[r] / rh;
        T sp;
        if (kind == K_ZERO) sp = T(0);
        else if (kind == K_NONNEG) sp = v > T(0) ? v : T(0);
        else sp = fmin(fmax(v, P.box_l[r]), P.box_u[r]);
        const T yn = q.y[r] + rh * (sh - sp);
        q.sn[r] = sp;
        q.yn[r] = yn;
        if (!finite_(yn) || !finite_(sp)) atomicOr(&q.flags[P.row_inst[r]], F_NONFINITE);
      }
    } else {
      const int64_t j = e - P.m_total;
      const T al = q.alpha[P.col_inst[j]];
      q.xn[j] = al * q.xt[j] + (T(1) - al) * q.x[j];
    }
  }
}

// a6 (SOC): one warp per cone {(t, u): ||u|| <= t}
template <class T, class V>
__global__ void k_soc_fwd(Prob<T, V> P, StepPtrs<T> q) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= P.nsoc) return;
  const int64_t r0 = P.soc_row0[w];
  const int32_t d = P.soc_dim[w];
  const int32_t inst = P.row_inst[r0];
  const T al = q.alpha[inst], rh = q.rho[r0];
  double nu2 = 0.0;
  for (int32_t i = 1 + lane; i < d; i += 32) {
    const int64_t r = r0 + i;
    const T v = al * q.st[r] + (T(1) - al) * q.s[r] + q.y[r] / rh;
    nu2 += (double)v * (double)v;
  }
  nu2 = warp_sum(nu2);
  const T t = al * q.st[r0] + (T(1) - al) * q.s[r0] + q.y[r0] / rh;
  const double nu = sqrt(nu2);
  int mode;  // 0 identity, 1 zero, 2 boundary projection
  if (nu <= (double)t) mode = 0;
  else if (nu <= -(double)t) mode = 1;
  else mode = 2;
  const T scale = mode == 2 ? (T)(0.5 * (1.0 + (double)t / nu)) : T(0);
  for (int32_t i = lane; i < d; i += 32) {
    const int64_t r = r0 + i;
    const T sh = al * q.st[r] + (T(1) - al) * q.s[r];
    const T v = sh + q.y[r] / rh;
    T sp;
    if (mode == 0) sp = v;
    else if (mode == 1) sp = T(0);
    else sp = scale * (i == 0 ? (T)nu : v);
    const T yn = q.y[r] + rh * (sh - sp);
    q.sn[r] = sp;
    q.yn[r] = yn;
    if (!finite_(yn)) atomicOr(&q.flags[inst], F_NONFINITE);
  }
}

// ---------------------------------------------------------------------------
// a9: residuals r_p = A x + s - b, r_d = P x + q - A'y (App. E; sign fixed by
// the fixed point of Sec. 2.2), per-instance ||r_p||^2, ||r_d||^2 and the
// objective 1/2 x'Px + q'x; one CTA per instance, double accumulation.
// ---------------------------------------------------------------------------
template <class T>
struct ResArgs {
  const T* x; const T* s; const T* y;
  T* rp; T* rd;        // stored residual vectors (may be null)
  double* rp2; double* rd2; double* obj; double* loss;  // [ninst] each, may be null
};

template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_residuals(Prob<T, V> P, ResArgs<T> a) {
  __shared__ double sm[3 * (NT / 32)];
  const int32_t inst = blockIdx.x;
  const int64_t c0 = P.col_off[inst], c1 = P.col_off[inst + 1];
  const int64_t r0 = P.row_off[inst], r1 = P.row_off[inst + 1];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t r = r0 + threadIdx.x; r < r1; r += NT) {
    T v = a.s[r] - P.b[r];
    for (int64_t e = P.A_rp[r]; e < P.A_rp[r + 1]; ++e) v += (T)ldv(P.A_v, e) * a.x[P.A_ci[e]];
    if (a.rp) a.rp[r] = v;
    acc[0] += (double)v * (double)v;
  }
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) {
    T px = T(0);
    if (P.P_rp) {
      for (int64_t e = P.P_rp[j]; e < P.P_rp[j + 1]; ++e) px += (T)ldv(P.P_v, e) * a.x[P.P_ci[e]];
    }
    T aty = T(0);
    for (int64_t e = P.AT_rp[j]; e < P.AT_rp[j + 1]; ++e) aty += (T)ldv(P.AT_v, e) * a.y[P.AT_ci[e]];
    const T v = px + P.q[j] - aty;
    if (a.rd) a.rd[j] = v;
    acc[1] += (double)v * (double)v;
    acc[2] += 0.5 * (double)a.x[j] * (double)px + (double)P.q[j] * (double)a.x[j];
  }
  block_sum<3>(acc, sm);
  if (threadIdx.x == 0) {
    if (a.rp2) a.rp2[inst] = acc[0];
    if (a.rd2) a.rd2[inst] = acc[1];
    if (a.obj) a.obj[inst] = acc[2];
    if (a.loss) a.loss[inst] = acc[0] + acc[1];
  }
}

// ---------------------------------------------------------------------------
// Log-residual meta-loss of Sec. 4: per instance
//   L = sum_{k=1..K} log(S_k),  S_k = ||r_d^k||^2 / ||r_d^0||^2 + ||r_p^k||^2 / ||r_p^0||^2
// with the k = 0 norms held constant; rd2 / rp2 hold ||r_d^k||^2, ||r_p^k||^2
// as [K + 1][ninst].  A term with a zero k = 0 norm is dropped and a step with
// S_k = 0 contributes nothing.  FP64 (one thread per instance).
__device__ __forceinline__ double logratio_sum(double a0, double b0, double ak, double bk) {
  return (a0 > 0.0 ? ak / a0 : 0.0) + (b0 > 0.0 ? bk / b0 : 0.0);
}

__global__ void k_logratio_loss(int32_t ninst, int32_t K, const double* __restrict__ rd2,
                                const double* __restrict__ rp2, double* __restrict__ loss) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  const double a0 = rd2[i], b0 = rp2[i];
  double L = 0.0;
  for (int32_t k = 1; k <= K; ++k) {
    const double S = logratio_sum(a0, b0, rd2[(int64_t)k * ninst + i], rp2[(int64_t)k * ninst + i]);
    if (S > 0.0) L += log(S);
  }
  loss[i] = L;
}

// weights of state k's cotangent: d(g log S_k)/d||r_d^k||^2 = g / (S_k a0),
// d/d||r_p^k||^2 = g / (S_k b0)
template <class T>
__global__ void k_logratio_w(int32_t ninst, int32_t k, const double* __restrict__ rd2,
                             const double* __restrict__ rp2, const double* __restrict__ gloss, T* wa, T* wb) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  const double a0 = rd2[i], b0 = rp2[i];
  const double S = logratio_sum(a0, b0, rd2[(int64_t)k * ninst + i], rp2[(int64_t)k * ninst + i]);
  const double g = gloss ? gloss[i] : 0.0;
  wa[i] = (T)((S > 0.0 && a0 > 0.0) ? g / (S * a0) : 0.0);
  wb[i] = (T)((S > 0.0 && b0 > 0.0) ? g / (S * b0) : 0.0);
}

// add state k's cotangent: x_bar += 2 wa P r_d + 2 wb A'r_p, s_bar += 2 wb r_p,
// y_bar -= 2 wa A r_d (r_p, r_d the state's residual vectors)
template <class T, class V>
__global__ void k_logratio_seed(Prob<T, V> P, const T* __restrict__ rp, const T* __restrict__ rd,
                                const T* __restrict__ wa, const T* __restrict__ wb, T* xb, T* sb, T* yb) {
  const int64_t tot = P.m_total + P.n_total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < P.m_total) {
      const int64_t r = e;
      const int32_t i = P.row_inst[r];
      const T a = wa[i], b = wb[i];
      T ard = T(0);
      if (a != T(0))
        for (int64_t q = P.A_rp[r]; q < P.A_rp[r + 1]; ++q) ard += (T)ldv(P.A_v, q) * rd[P.A_ci[q]];
      yb[r] -= T(2) * a * ard;
      sb[r] += T(2) * b * rp[r];
    } else {
      const int64_t j = e - P.m_total;
      const int32_t i = P.col_inst[j];
      const T a = wa[i], b = wb[i];
      T acc = T(0);
      if (b != T(0))
        for (int64_t q = P.AT_rp[j]; q < P.AT_rp[j + 1]; ++q) acc += b * (T)ldv(P.AT_v, q) * rp[P.AT_ci[q]];
      if (P.P_rp && a != T(0))
        for (int64_t q = P.P_rp[j]; q < P.P_rp[j + 1]; ++q) acc += a * P.P_v[q] * rd[P.P_ci[q]];
      xb[j] += T(2) * acc;
    }
  }
}

// ---------------------------------------------------------------------------
// b1: loss backward.  d/dx = 2 (A'r_p + P r_d), d/ds = 2 r_p, d/dy = -2 A r_d,
// each times the per-instance loss cotangent, plus the caller's cotangents.
// ---------------------------------------------------------------------------
template <class T>
struct SeedArgs {
  const T* rp; const T* rd; const double* gloss;   // gloss may be null
  const T* gx; const T* gs; const T* gy;           // may be null
  T* xb; T* sb; T* yb;
};

template <class T, class V>
__global__ void k_loss_seed(Prob<T, V> P, SeedArgs<T> a) {
  const int64_t tot = P.m_total + P.n_total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < P.m_total) {
      const int64_t r = e;
      const T g = a.gloss ? (T)a.gloss[P.row_inst[r]] : T(0);
      T ys = a.gy ? a.gy[r] : T(0);
      T ss = a.gs ? a.gs[r] : T(0);
      if (a.gloss) {
        T ard = T(0);
        for (int64_t k = P.A_rp[r]; k < P.A_rp[r + 1]; ++k) ard += (T)ldv(P.A_v, k) * a.rd[P.A_ci[k]];
        ys -= T(2) * g * ard;
        ss += T(2) * g * a.rp[r];
      }
      a.yb[r] = ys;
      a.sb[r] = ss;
    } else {
      const int64_t j = e - P.m_total;
      T xs = a.gx ? a.gx[j] : T(0);
      if (a.gloss) {
        const T g = (T)a.gloss[P.col_inst[j]];
        T acc = T(0);
        for (int64_t k = P.AT_rp[j]; k < P.AT_rp[j + 1]; ++k) acc += (T)ldv(P.AT_v, k) * a.rp[P.AT_ci[k]];
        if (P.P_rp) {
          for (int64_t k = P.P_rp[j]; k < P.P_rp[j + 1]; ++k) acc += (T)ldv(P.P_v, k) * a.rd[P.P_ci[k]];
        }
        xs += T(2) * g * acc;
      }
      a.xb[j] = xs;
    }
  }
}

// ---------------------------------------------------------------------------
// Reverse pass of one iteration.  Cotangents of z^{k+1} come in (xb, sb, yb);
// those of z^k go out (xb2, sb2, yb2), together with rho-bar (per row, before
// the rectification adjoint) and alpha-bar (per instance).
// ---------------------------------------------------------------------------
template <class T>
struct BwdPtrs {
  const T* x; const T* s; const T* y;   // z^k
  const T* sn;                          // s^{k+1}
  const T* rho; const T* alpha; double sigma;
  const T* xt; const T* st;             // tape
  const T* lam; const T* U;
  const T* xb; const T* sb; const T* yb;   // cotangents of z^{k+1}
  T* xb2; T* sb2; T* yb2;                  // cotangents of z^k
  T* gproj;  // [m_total] cotangent reaching the projection output
  T* vbar;   // [m_total] cotangent of the projection input v
  T* adjrhs; // [n_total] -x~bar
  T* lamt;       // [n_total] adjoint solution lambda~
  const T* dinv; // [n_total] inverse diagonal of M (diagonal-M instances)
  T* grho;   // [m_total] rho-bar of this step (unrectified later)
  T* galpha; // [ninst]
  int32_t* flags;
  double dk_tau;
};

// b2 (first half) + b3 separable: g = s+bar - rho y+bar; vbar = mask(v) g
template <class T, class V>
__global__ void k_bwd_gproj(Prob<T, V> P, BwdPtrs<T> q) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < P.m_total;
       r += (int64_t)gridDim.x * blockDim.x) {
    const T rh = q.rho[r];
    const T g = q.sb[r] - rh * q.yb[r];
    q.gproj[r] = g;
    const uint8_t kind = P.row_kind[r];
    if (kind <= K_BOX) {
      const T al = q.alpha[P.row_inst[r]];
      const T v = al * q.st[r] + (T(1) - al) * q.s[r] + q.y[r] / rh;
      bool pass;
      if (kind == K_ZERO) pass = false;
      else if (kind == K_NONNEG) pass = v > T(0);
      else pass = (v > P.box_l[r]) && (v < P.box_u[r]);
      q.vbar[r] = pass ? g : T(0);
    }
  }
}

// b3 (SOC): vbar = J' g with the closed-form Jacobian of the SOC projection
template <class T, class V>
__global__ void k_soc_bwd(Prob<T, V> P, BwdPtrs<T> q) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= P.nsoc) return;
  const int64_t r0 = P.soc_row0[w];
  const int32_t d = P.soc_dim[w];
  const int32_t inst = P.row_inst[r0];
  const T al = q.alpha[inst], rh = q.rho[r0];
  double nu2 = 0.0, ug = 0.0;
  for (int32_t i = 1 + lane; i < d; i += 32) {
    const int64_t r = r0 + i;
    const T v = al * q.st[r] + (T(1) - al) * q.s[r] + q.y[r] / rh;
    nu2 += (double)v * (double)v;
    ug += (double)v * (double)q.gproj[r];
  }
  nu2 = warp_sum(nu2);
  ug = warp_sum(ug);
  const T t = al * q.st[r0] + (T(1) - al) * q.s[r0] + q.y[r0] / rh;
  const double nu = sqrt(nu2);
  int mode;
  if (nu <= (double)t) mode = 0;
  else if (nu <= -(double)t) mode = 1;
  else mode = 2;
  const double g0 = (double)q.gproj[r0];
  const double uhg = mode == 2 ? ug / nu : 0.0;     // u^' g_u
  const double tn = mode == 2 ? (double)t / nu : 0.0;
  for (int32_t i = lane; i < d; i += 32) {
    const int64_t r = r0 + i;
    T out;
    if (mode == 0) out = q.gproj[r];
    else if (mode == 1) out = T(0);
    else if (i == 0) out = (T)(0.5 * (g0 + uhg));
    else {
      const T v = al * q.st[r] + (T(1) - al) * q.s[r] + q.y[r] / rh;
      const double uh = (double)v / nu;
      out = (T)(0.5 * (g0 * uh + (1.0 + tn) * (double)q.gproj[r] - tn * uh * uhg));
    }
    q.vbar[r] = out;
  }
}

// b2 (rest) + b4: per instance (one CTA), fixed-order alpha-bar reduction.
//   shat_bar = rho y+bar + vbar ;  s~bar = alpha shat_bar
//   ybar_part = y+bar + vbar / rho ; sbar_part = (1-alpha) shat_bar
//   rhobar_part = y+bar (shat - s+) - vbar y / rho^2
//   x~bar = alpha x+bar - A' s~bar ; xbar_part = (1-alpha) x+bar
//   alpha_bar = <shat_bar, s~ - s> + <x+bar, x~ - x>
// The rows' s~bar goes to vbar (one gather per A' entry in the column loop
// instead of three); 512 threads so that the largest instances take few
// passes of the dependent row-pointer -> index -> value chain.
// A thread's running sum of products a*b, for the per-instance double
// reductions of the backward.  FP32: each product split exactly into
// p + e by a fused multiply-add (TwoProduct), both added with Neumaier's
// compensated summation in FP32, converted to double once -- the double
// accumulation of the exact products to within a few units of 2^-48 of the
// sum of the magnitudes, without an FP64 operation per element (slow on this
// part).  FP64: the plain double sum.
template <class T>
struct CompSum {
  double d = 0.0;
  __device__ __forceinline__ void add_prod(T a, T b) { d += (double)a * (double)b; }
  __device__ __forceinline__ double value() const { return d; }
};
template <>
struct CompSum<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add1(float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    add1(p);
    c += e;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_bwd_relax(Prob<T, V> P, BwdPtrs<T> q) {
  __shared__ double sm[NT / 32];
  const int32_t inst = blockIdx.x;
  const int64_t c0 = P.col_off[inst], c1 = P.col_off[inst + 1];
  const int64_t r0 = P.row_off[inst], r1 = P.row_off[inst + 1];
  const T al = q.alpha[inst];
  const bool diag = P.diag_inst[inst] != 0;
  CompSum<T> acc0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += NT) {
    const T rh = q.rho[r];
    const T yb = q.yb[r], vb = q.vbar[r];
    const T shb = rh * yb + vb;
    const T s = q.s[r], st = q.st[r], y = q.y[r];
    const T sh = al * st + (T(1) - al) * s;
    q.yb2[r] = yb + vb / rh;
    q.sb2[r] = (T(1) - al) * shb;
    q.grho[r] = yb * (sh - q.sn[r]) - vb * y / (rh * rh);
    acc0.add_prod(shb, st - s);
    if (!finite_(shb)) atomicOr(&q.flags[inst], F_NONFINITE);
    q.vbar[r] = al * shb;   // s~bar, read back by the A' product below (vbar is dead after this kernel)
  }
  __syncthreads();          // the instance's rows are all this CTA's: its own writes are visible
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) {
    const T xb = q.xb[j];
    T acc2 = al * xb;
    for (int64_t e = P.AT_rp[j]; e < P.AT_rp[j + 1]; ++e) acc2 -= (T)ldv(P.AT_v, e) * q.vbar[P.AT_ci[e]];
    if (diag) q.lamt[j] = -acc2 * q.dinv[j];
    else q.adjrhs[j] = -acc2;
    q.xb2[j] = (T(1) - al) * xb;
    acc0.add_prod(xb, q.xt[j] - q.x[j]);
  }
  double acc[1] = {acc0.value()};
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) q.galpha[inst] = (T)acc[0];
}

// b5 (after the adjoint CG): w = A lambda~;  rho-bar += w o (s - s~)
// (the implicit rule (A lam)(A x~) plus the RHS chain), y-bar -= w,
// s-bar += rho w, x-bar -= sigma lambda~.
template <class T, class V>
__global__ void k_bwd_solve(Prob<T, V> P, BwdPtrs<T> q) {
  const int64_t tot = P.m_total + P.n_total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < P.m_total) {
      const int64_t r = e;
      T w = T(0);
      for (int64_t k = P.A_rp[r]; k < P.A_rp[r + 1]; ++k) w += (T)ldv(P.A_v, k) * q.lamt[P.A_ci[k]];
      q.grho[r] += w * (q.s[r] - q.st[r]);
      q.yb2[r] -= w;
      q.sb2[r] += q.rho[r] * w;
    } else {
      const int64_t j = e - P.m_total;
      q.xb2[j] -= (T)q.sigma * q.lamt[j];
    }
  }
}

// b6: adjoint of the rectification over all K steps: every row of a SOC/PSD
// block receives the block mean of rho-bar.  L lanes per (step, block), as
// k_rho_rectify.
template <class T, class V, int L>
__global__ void k_rect_adjoint(Prob<T, V> P, int32_t K, T* __restrict__ g) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / L;
  const int lane = threadIdx.x % L;
  if (w >= (int64_t)K * P.nrect) return;   // whole lane groups
  const int32_t k = (int32_t)(w / P.nrect), c = (int32_t)(w % P.nrect);
  T* dst = g + (int64_t)k * P.m_total + P.rect_row0[c];
  const int32_t nr = P.rect_rows[c];
  double acc = 0.0;
  for (int32_t i = lane; i < nr; i += L) acc += (double)dst[i];
  acc = group_sum<L>(acc);
  __syncwarp(group_mask<L>());             // the group's reads before its writes
  const T mean = (T)(acc / (double)nr);
  for (int32_t i = lane; i < nr; i += L) dst[i] = mean;
}

// ---------------------------------------------------------------------------
// standalone solve helpers: the Jacobi preconditioner from a caller's CSR
// (the diagonal of P is looked up in its rows) and an identity schedule
// ---------------------------------------------------------------------------
template <class T, class V>
__global__ void k_precond_csr(Prob<T, V> P, double sigma, const T* __restrict__ rho,
                              T* __restrict__ dinv) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.n_total;
       j += (int64_t)gridDim.x * blockDim.x) {
    T acc = (T)sigma;
    if (P.P_rp) {
      for (int64_t e = P.P_rp[j]; e < P.P_rp[j + 1]; ++e)
        if (P.P_ci[e] == j) acc += (T)ldv(P.P_v, e);
    }
    for (int64_t e = P.AT_rp[j]; e < P.AT_rp[j + 1]; ++e) {
      const T a = (T)ldv(P.AT_v, e);
      acc += a * a * rho[P.AT_ci[e]];
    }
    dinv[j] = T(1) / acc;
  }
}

__global__ void k_iota(int32_t n, int32_t* __restrict__ out) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = i;
}

// ---------------------------------------------------------------------------
// parameter maps for per-iteration learnable scalars
// ---------------------------------------------------------------------------
template <class T, class V>
__global__ void k_rho_from_log(Prob<T, V> P, int32_t K, const double* __restrict__ logr,
                               double eq_scale, T* __restrict__ rho) {
  // blockIdx.y = step k: exp(log rho_k) once per thread, not per entry
  const int32_t k = blockIdx.y;
  const double base = exp(logr[k]);
  const T b1 = (T)base, beq = (T)(eq_scale * base);
  T* __restrict__ out = rho + (int64_t)k * P.m_total;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < P.m_total;
       r += (int64_t)gridDim.x * blockDim.x)
    out[r] = P.row_kind[r] == K_ZERO ? beq : b1;
}

// glog[k] = sum_r grho[k][r] rho[k][r]; one CTA per step, fixed order.
template <class T, int NT>
__global__ void __launch_bounds__(NT) k_rowsum_prod(int64_t m, const T* __restrict__ a,
                                                    const T* __restrict__ b,
                                                    double* __restrict__ out) {
  __shared__ double sm[NT / 32];
  const int32_t k = blockIdx.x;
  double acc[1] = {0.0};
  const T* ak = a + (int64_t)k * m;
  const T* bk = b ? b + (int64_t)k * m : nullptr;
  for (int64_t r = threadIdx.x; r < m; r += NT) acc[0] += (double)ak[r] * (bk ? (double)bk[r] : 1.0);
  block_sum<1>(acc, sm);
  if (threadIdx.x == 0) out[k] = acc[0];
}

template <class T>
__global__ void k_broadcast(int32_t K, int32_t w, const double* __restrict__ src,
                            T* __restrict__ dst) {
  const int64_t tot = (int64_t)K * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (T)src[e / w];
}

// ---------------------------------------------------------------------------
// Solve to tolerance (the vanilla COSMO baseline of Sec. 4 / App. D): KKT
// residual infinity norms, the stop test and OSQP-style residual balancing
// of one scalar rho per instance.
// ---------------------------------------------------------------------------

// per instance (one CTA): ||Ax + s - b||, ||Ax||, ||s||, ||b||,
// ||Px + q - A'y||, ||Px||, ||q||, ||A'y||, all infinity norms, into
// nrm[k * ninst + inst] (FP64; the maxima are exact in any order)
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_kkt_inf(Prob<T, V> P, const T* __restrict__ x, const T* __restrict__ s,
                                                const T* __restrict__ y, double* __restrict__ nrm) {
  __shared__ double sm[8][NT / 32];
  const int32_t inst = blockIdx.x;
  const int64_t c0 = P.col_off[inst], c1 = P.col_off[inst + 1];
  const int64_t r0 = P.row_off[inst], r1 = P.row_off[inst + 1];
  // maxima of |.| in the iterate type (exact: a maximum does not round), widened at the end
  T v[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  for (int64_t r = r0 + threadIdx.x; r < r1; r += NT) {
    T ax = T(0);
    for (int64_t e = P.A_rp[r]; e < P.A_rp[r + 1]; ++e) ax += (T)ldv(P.A_v, e) * x[P.A_ci[e]];
    v[0] = fmax(v[0], fabs(ax + s[r] - P.b[r]));
    v[1] = fmax(v[1], fabs(ax));
    v[2] = fmax(v[2], fabs(s[r]));
    v[3] = fmax(v[3], fabs(P.b[r]));
  }
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) {
    T px = T(0), aty = T(0);
    if (P.P_rp)
      for (int64_t e = P.P_rp[j]; e < P.P_rp[j + 1]; ++e) px += (T)ldv(P.P_v, e) * x[P.P_ci[e]];
    for (int64_t e = P.AT_rp[j]; e < P.AT_rp[j + 1]; ++e) aty += (T)ldv(P.AT_v, e) * y[P.AT_ci[e]];
    v[4] = fmax(v[4], fabs(px + P.q[j] - aty));
    v[5] = fmax(v[5], fabs(px));
    v[6] = fmax(v[6], fabs(P.q[j]));
    v[7] = fmax(v[7], fabs(aty));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = fmax(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    if (lane == 0) sm[k][w] = (double)v[k];
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double mx = 0.0;
    for (int q = 0; q < NT / 32; ++q) mx = fmax(mx, sm[threadIdx.x][q]);
    nrm[(int64_t)threadIdx.x * P.ninst + inst] = mx;
  }
}

struct SolveCtl {
  double eps;            // stop when both normalised residuals are <= eps
  double tol;            // rebalance when the ratio leaves [1/tol, tol]
  double rho_min, rho_max;
  int32_t it;            // iterations done
  int32_t rebalance;     // 1: rebalance at this check
};

// one thread per instance: normalised residuals rbar_p = ||r_p|| / max(||Ax||,
// ||s||, ||b||), rbar_d = ||r_d|| / max(||Px||, ||q||, ||A'y||) (a zero
// scale counts as 1); first iteration count at which both are <= eps; for
// unconverged instances at a rebalancing check rho <- rho sqrt(rbar_p /
// rbar_d) when that factor leaves [1/tol, tol], clipped to [rho_min,
// rho_max]; *running counts the unconverged instances
__global__ void k_solve_update(int32_t ninst, const double* __restrict__ nrm, SolveCtl c, double* __restrict__ rho,
                               int32_t* __restrict__ conv_it, double* __restrict__ rbp, double* __restrict__ rbd,
                               int32_t* __restrict__ running) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  auto at = [&](int k) { return nrm[(int64_t)k * ninst + i]; };
  const double sp = fmax(fmax(at(1), at(2)), at(3)), sd = fmax(fmax(at(5), at(6)), at(7));
  const double p = at(0) / (sp > 0.0 ? sp : 1.0), d = at(4) / (sd > 0.0 ? sd : 1.0);
  rbp[i] = p;
  rbd[i] = d;
  const bool done = p <= c.eps && d <= c.eps;
  if (done && conv_it[i] < 0) conv_it[i] = c.it;
  if (conv_it[i] >= 0) return;
  atomicAdd(running, 1);
  if (c.rebalance && p > 0.0 && d > 0.0) {
    const double f = sqrt(p / d);
    if (f > c.tol || f < 1.0 / c.tol) rho[i] = fmin(fmax(rho[i] * f, c.rho_min), c.rho_max);
  }
}

// rho rows of K steps from the instances' scalars (x eq on zero-cone rows),
// alpha of K steps
template <class T, class V>
__global__ void k_solve_fill(Prob<T, V> P, int32_t K, const double* __restrict__ rho, double eq, double alpha,
                             T* __restrict__ rho_rows, T* __restrict__ alpha_k) {
  const int64_t tot = (int64_t)K * P.m_total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % P.m_total;
    const double v = rho[P.row_inst[r]] * (P.row_kind[r] == K_ZERO ? eq : 1.0);
    rho_rows[e] = (T)v;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)K * P.ninst;
       e += (int64_t)gridDim.x * blockDim.x)
    alpha_k[e] = (T)alpha;
}

}  // namespace cosmo
