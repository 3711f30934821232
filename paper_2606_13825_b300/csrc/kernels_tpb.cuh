// PSD projection (a7, a8) and its Daleckii-Krein backward (b3) for blocks of
// order p <= 8, one block per THREAD (Sec. 2.4, Eqs. psd-proj,
// psd-cotangent-dk, lowner).  Batches of many tiny blocks (covariance
// steering: 41 blocks of orders 4..8 per instance, 20,992 in the workload)
// would otherwise give each block a whole CTA whose barriers, reductions and
// 128-row tensor-core tiles it cannot fill.  A thread keeps its block's
// matrices in shared memory, interleaved across the CTA (entry e of thread
// t at [e * NT + t]), so the threads of a warp touch 32 consecutive words
// and never conflict; no barrier is needed.
//
// Forward, per block: S from the relaxed iterate (as the CTA kernels),
// warm start B = V' S V from the previous step's eigenvectors, cyclic Jacobi
// sweeps in row order with the CTA kernels' rotation (jt_rotation, the same
// threshold and stopping rules), then the refinement of reading c-22 (one
// Newton-Schulz step, the Rayleigh-Ritz matrix of S again, eigenvalues as
// its diagonal, Pi = V'(max(L, 0) + G o E)V with the first-order correction
// of the off-diagonal E), the eigen tape and the fused dual update.
// Backward: S_bar = U (L o (U' G U)) U' with the Loewner matrix of max(x, 0)
// decided as in the tensor-core kernel: 1 / 0 / 1/2 for same-sign pairs
// without a division, l+ / (l+ - l-) in the iterate type for mixed-sign pairs
// certainly outside the tie band, the FP64 rule of reading c-4 otherwise.
#pragma once

#include "common.cuh"
#include "kernels_jt.cuh"
#include "kernels_psd.cuh"

namespace cosmo {

constexpr int TPB_MAXP = 8;
constexpr int TPB_NT = 64;      // threads (blocks) per CTA

// one thread's p x p matrix (row stride TPB_MAXP) in a buffer of NT threads
template <class T, int NT>
struct TpbMat {
  T* b;
  __device__ __forceinline__ T& operator()(int i, int j) const { return b[(i * TPB_MAXP + j) * NT]; }
};

template <class T>
__host__ __device__ constexpr size_t tpb_smem(int nt) {
  return (size_t)3 * TPB_MAXP * TPB_MAXP * nt * sizeof(T);
}

// C = A B (p x p), C distinct from A and B.  The TPB_MAXP outputs of a row
// are formed together (their FMA chains interleave; entries beyond p are
// skipped by predicate); each sum runs over k in order.
template <class T, int NT>
__device__ __forceinline__ void tpb_mm(int p, TpbMat<T, NT> A, TpbMat<T, NT> B, TpbMat<T, NT> C) {
  for (int i = 0; i < p; ++i) {
    T acc[TPB_MAXP];
#pragma unroll
    for (int j = 0; j < TPB_MAXP; ++j) acc[j] = T(0);
    for (int k = 0; k < p; ++k) {
      const T a = A(i, k);
#pragma unroll
      for (int j = 0; j < TPB_MAXP; ++j)
        if (j < p) acc[j] = fma(a, B(k, j), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < TPB_MAXP; ++j)
      if (j < p) C(i, j) = acc[j];
  }
}
// C = A B'
template <class T, int NT>
__device__ __forceinline__ void tpb_mmt(int p, TpbMat<T, NT> A, TpbMat<T, NT> B, TpbMat<T, NT> C) {
  for (int i = 0; i < p; ++i) {
    T acc[TPB_MAXP];
#pragma unroll
    for (int j = 0; j < TPB_MAXP; ++j) acc[j] = T(0);
    for (int k = 0; k < p; ++k) {
      const T a = A(i, k);
#pragma unroll
      for (int j = 0; j < TPB_MAXP; ++j)
        if (j < p) acc[j] = fma(a, B(j, k), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < TPB_MAXP; ++j)
      if (j < p) C(i, j) = acc[j];
  }
}
// C = A' B
template <class T, int NT>
__device__ __forceinline__ void tpb_mtm(int p, TpbMat<T, NT> A, TpbMat<T, NT> B, TpbMat<T, NT> C) {
  for (int i = 0; i < p; ++i) {
    T acc[TPB_MAXP];
#pragma unroll
    for (int j = 0; j < TPB_MAXP; ++j) acc[j] = T(0);
    for (int k = 0; k < p; ++k) {
      const T a = A(k, i);
#pragma unroll
      for (int j = 0; j < TPB_MAXP; ++j)
        if (j < p) acc[j] = fma(a, B(k, j), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < TPB_MAXP; ++j)
      if (j < p) C(i, j) = acc[j];
  }
}

// sum over the warp's converged lanes of one counter, added by the first of them
__device__ __forceinline__ void tpb_count(unsigned long long* ctr, unsigned v) {
  const unsigned mask = __activemask();
  const unsigned s = __reduce_add_sync(mask, v);
  if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(ctr, (unsigned long long)s);
}

template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_psd_fwd_tpb(Prob<T, V> P, PsdIterIO<T> io, T* lam_slot, T* U_slot,
                                                    double tol, int max_sweeps, int32_t* flags, int sched_off,
                                                    int count, unsigned long long* stats, const T* U_prev) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int q = blockIdx.x * NT + threadIdx.x;
  if (q >= count) return;                      // no barrier below: threads are independent
  T* base = reinterpret_cast<T*>(smraw) + threadIdx.x;
  const TpbMat<T, NT> A{base}, Vt{base + TPB_MAXP * TPB_MAXP * NT}, W{base + 2 * TPB_MAXP * TPB_MAXP * NT};
  const int blk = P.psd_sched[sched_off + q];
  const int p = P.psd_p[blk];
  const int64_t row0 = P.psd_row0[blk];
  const int inst = io.row_inst[row0];
  const T al = io.alpha[inst], rh = io.rho[row0];
  auto load_S = [&](TpbMat<T, NT> S) {
    for (int j = 0; j < p; ++j)
      for (int i = 0; i <= j; ++i) {
        const int64_t r = row0 + j * (j + 1) / 2 + i;
        T v = al * io.st[r] + (T(1) - al) * io.s[r] + io.y[r] / rh;
        if (i != j) v *= (T)kInvSqrt2;
        S(i, j) = v;
        S(j, i) = v;
      }
  };
  // Vt: rows are eigenvectors (previous step's, or the identity)
  if (U_prev) {
    const T* Up = U_prev + P.psd_uoff[blk];
    for (int k = 0; k < p; ++k)
      for (int i = 0; i < p; ++i) Vt(k, i) = Up[k * p + i];
    load_S(W);
    tpb_mm<T, NT>(p, Vt, W, A);                // A = Vt S
    tpb_mmt<T, NT>(p, A, Vt, W);               // W = Vt S Vt'
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) A(i, j) = W(i, j);
  } else {
    for (int k = 0; k < p; ++k)
      for (int i = 0; i < p; ++i) Vt(k, i) = k == i ? T(1) : T(0);
    load_S(A);
  }
  // cyclic Jacobi (row order), the stopping rules of the CTA kernels
  const double tol_eff = fmax(tol, 4.0 * Eps<T>::v * sqrt((double)p));
  const double tol2 = tol_eff * tol_eff;
  double prev_off2 = 0.0;
  int sweeps = -max_sweeps;
  for (int sweep = 0;; ++sweep) {
    T off = T(0), dia = T(0);
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) {
        const T a = A(i, j);
        if (i == j) dia += a * a;
        else off += a * a;
      }
    const double off2 = off, tot2 = (double)off + (double)dia;
    if (off2 <= tol2 * tot2 || (sweep >= 5 && off2 > 0.5 * prev_off2)) { sweeps = sweep; break; }
    if (sweep >= max_sweeps) break;
    prev_off2 = off2;
    const T thresh = (T)(tol_eff * sqrt(tot2) / (4.0 * p));
    for (int a = 0; a < p - 1; ++a)
      for (int b = a + 1; b < p; ++b) {
        JtQuad<T> x;
        x.aa = A(a, a); x.ab = A(a, b); x.ba = x.ab; x.bb = A(b, b);
        const JtRot<T> r = jt_rotation(x.aa, x.ab, x.bb, thresh);
        if (r.s == T(0)) continue;
#pragma unroll
        for (int k = 0; k < TPB_MAXP; ++k) {
          if (k >= p || k == a || k == b) continue;
          const T ka = A(k, a), kb = A(k, b);
          const T na = jt_cms(r.c, r.s, ka, kb), nb = jt_spc(r.c, r.s, ka, kb);
          A(k, a) = na; A(a, k) = na;
          A(k, b) = nb; A(b, k) = nb;
        }
        A(a, a) = jt_diag_a(x, r);
        A(b, b) = jt_diag_b(x, r);
        A(a, b) = T(0); A(b, a) = T(0);
#pragma unroll
        for (int k = 0; k < TPB_MAXP; ++k) {
          if (k >= p) continue;
          const T va = Vt(a, k), vb = Vt(b, k);
          Vt(a, k) = jt_cms(r.c, r.s, va, vb);
          Vt(b, k) = jt_spc(r.c, r.s, va, vb);
        }
      }
  }
  if (sweeps < 0) atomicOr(&flags[inst], F_EIG_CAP);
  if (stats) {
    tpb_count(&stats[0], (unsigned)(sweeps < 0 ? -sweeps : sweeps));
    tpb_count(&stats[1], 1u);
  }
  // refinement: Newton-Schulz, Vt <- 1.5 Vt - 0.5 (Vt Vt') Vt
  tpb_mmt<T, NT>(p, Vt, Vt, A);
  tpb_mm<T, NT>(p, A, Vt, W);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) Vt(i, j) = T(1.5) * Vt(i, j) - T(0.5) * W(i, j);
  // Rayleigh-Ritz: X = Vt S, eigenvalues L_i = (X Vt')_ii, R = X Vt'
  load_S(W);
  tpb_mm<T, NT>(p, Vt, W, A);                  // A = X
  T lam[TPB_MAXP];
#pragma unroll
  for (int i = 0; i < TPB_MAXP; ++i) {
    T acc = T(0);
    if (i < p)
      for (int k = 0; k < p; ++k) acc = fma(Vt(i, k), A(i, k), acc);
    lam[i] = acc;
  }
  tpb_mmt<T, NT>(p, A, Vt, W);                 // W = R
  // M = max(L, 0) + G o E (E the off-diagonal of R), into W
#pragma unroll
  for (int i = 0; i < TPB_MAXP; ++i)
#pragma unroll
    for (int j = 0; j < TPB_MAXP; ++j) {
      if (i >= p || j >= p) continue;
      const T li = lam[i], lj = lam[j];
      if (i == j) {
        W(i, i) = li > T(0) ? li : T(0);
      } else {
        const bool pi = li > T(0), pj = lj > T(0);
        T g;
        if (pi && pj) g = T(1);
        else if (!pi && !pj) g = T(0);
        else {
          const T lp = pi ? li : lj, ln = pi ? lj : li;
          g = lp / (lp - ln);
        }
        W(i, j) = g * W(i, j);
      }
    }
  // Pi = Vt' M Vt: A = M Vt, then Pi(i, j) = sum_k Vt(k, i) A(k, j)
  tpb_mm<T, NT>(p, W, Vt, A);
  T* lam_out = lam_slot + P.psd_loff[blk];
  T* U = U_slot + P.psd_uoff[blk];
#pragma unroll
  for (int i = 0; i < TPB_MAXP; ++i)
    if (i < p) lam_out[i] = lam[i];
  for (int k = 0; k < p; ++k)
    for (int i = 0; i < p; ++i) U[k * p + i] = Vt(k, i);
  bool bad = false;
  for (int j = 0; j < p; ++j)
    for (int i = 0; i <= j; ++i) {
      T out = T(0);
      for (int k = 0; k < p; ++k) out = fma(Vt(k, i), A(k, j), out);
      if (i != j) out *= (T)kSqrt2;
      const int64_t r = row0 + j * (j + 1) / 2 + i;
      const T sh = al * io.st[r] + (T(1) - al) * io.s[r];
      const T yn = io.y[r] + rh * (sh - out);
      io.sn[r] = out;
      io.yn[r] = yn;
      bad = bad || !finite_(yn);
    }
  if (bad) atomicOr(&flags[inst], F_NONFINITE);
}

// b3: vbar = svec(U (L o (U' smat(g) U)) U') per block, one block per thread
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_psd_bwd_tpb(Prob<T, V> P, PsdBwdIO<T> io, const T* lam_slot,
                                                    const T* U_slot, double dk_tau_rel, int sched_off, int count) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int q = blockIdx.x * NT + threadIdx.x;
  if (q >= count) return;
  T* base = reinterpret_cast<T*>(smraw) + threadIdx.x;
  const TpbMat<T, NT> Us{base}, G{base + TPB_MAXP * TPB_MAXP * NT}, W{base + 2 * TPB_MAXP * TPB_MAXP * NT};
  const int blk = P.psd_sched[sched_off + q];
  const int p = P.psd_p[blk];
  const int64_t row0 = P.psd_row0[blk];
  const T* lamp = lam_slot + P.psd_loff[blk];
  const T* U = U_slot + P.psd_uoff[blk];
  T lam[TPB_MAXP];
  double lmax = 0.0;
#pragma unroll
  for (int k = 0; k < TPB_MAXP; ++k) {
    lam[k] = k < p ? lamp[k] : T(0);
    lmax = fmax(lmax, fabs((double)lam[k]));
  }
  const double tau = dk_tau_rel * fmax(1.0, lmax);
  for (int k = 0; k < p; ++k)
    for (int i = 0; i < p; ++i) Us(i, k) = U[k * p + i];      // Us(i, k): component i of vector k
  for (int j = 0; j < p; ++j)
    for (int i = 0; i <= j; ++i) {
      T v = io.g[row0 + j * (j + 1) / 2 + i];
      if (i != j) v *= (T)kInvSqrt2;
      G(i, j) = v;
      G(j, i) = v;
    }
  tpb_mtm<T, NT>(p, Us, G, W);                 // W = U' G
  tpb_mm<T, NT>(p, W, Us, G);                  // G = U' G U
#pragma unroll
  for (int k = 0; k < TPB_MAXP; ++k)
#pragma unroll
    for (int l = 0; l < TPB_MAXP; ++l) {
      if (k >= p || l >= p) continue;
      const T lk = lam[k], ll = lam[l];
      const bool pk = lk > T(0), pl = ll > T(0);
      T w;
      if (pk && pl) w = T(1);
      else if (!pk && !pl) w = (lk == T(0) && ll == T(0)) ? T(0.5) : T(0);
      else if (fabs((double)lk - (double)ll) > tau) {
        const T lp = pk ? lk : ll, ln = pk ? ll : lk;
        w = lp / (lp - ln);
      } else {
        w = (T)loewner_relu((double)lk, (double)ll, tau);
      }
      G(k, l) = w * G(k, l);
    }
  tpb_mm<T, NT>(p, Us, G, W);                  // W = U (L o (U' G U))
  for (int j = 0; j < p; ++j)
    for (int i = 0; i <= j; ++i) {
      T acc = T(0);
      for (int l = 0; l < p; ++l) acc = fma(W(i, l), Us(j, l), acc);
      if (i != j) acc *= (T)kSqrt2;
      io.vbar[row0 + j * (j + 1) / 2 + i] = acc;
    }
}

}  // namespace cosmo
