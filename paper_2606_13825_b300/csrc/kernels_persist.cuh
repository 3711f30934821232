// Persistent forward of the unrolled iteration (Sec. 2.2, Eqs.
// cosmo_linear_system .. cosmo_projection) for batches in which every
// instance has a diagonal reduced system and exactly one PSD block, its
// other rows being zero, nonnegative or box rows (max-cut: X_ii = 1 and one
// PSD cone).  One CTA owns one instance for all steps of a segment: per step
// it forms the right-hand side and x~ = D^-1 xi for the instance's columns
// (a3/a4), then s~ = b - A x~, the relaxation and projection of the
// separable rows and the relaxed x (a5, a6, a8), then the PSD projection
// with the fused dual update (a7, a8: jt2_project), and goes on to the next
// step without leaving the kernel.  Instances never read one another's
// rows, so no grid-wide wait is needed, and one launch per PSD size class
// covers the whole segment.  The per-element arithmetic is that of k_rhs,
// k_post and k_psd_fwd_jt2 in the same order, so the results equal the
// per-step launches bit for bit.
//
// Measured on the batched max-cut workload (256 instances, three size
// classes): slower than the per-step launches in graph mode (15.0 against
// 13.0 ms per forward), about equal with direct launches.  Each CTA keeps
// its SM for the whole segment, so the largest blocks share SMs with the
// smaller classes' CTAs for the first third of the steps, where the
// per-step launches place the classes afresh at every step; and the step
// loop around the inlined projection adds register spills to the Jacobi
// rounds (ptxas: 352 / 496 spill bytes against 108 / 352), while moving the
// phases into non-inlined functions spilled more (436 / 1132 in the
// projection).  Hence an option (fwd_persistent), off by default.
#pragma once

#include "common.cuh"
#include "kernels_jt2.cuh"
#include "kernels_vec.cuh"

namespace cosmo {

template <class T>
struct PersistArgs {
  int32_t k0, k1;             // steps [k0, k1) of a segment; step k uses slot k - k0
  const T* rho;               // rectified rho of every step [K][m_total]
  const T* alpha;             // [K][ninst]
  const double* sigma;        // [K]
  const T* dinv;              // Jacobi inverse diagonal of every step [K][n_total]
  T* xs; T* ss; T* ys;        // state slots [(c + 1)][n_total | m_total]
  T* xts; T* sts;             // tape x~, s~ [c][n_total | m_total]
  T* lams; T* Us;             // eigen tape [c][sum p], [c][sum p^2]
  const T* U_warm;            // eigenvectors that warm-start step k0 (null: cold start at k0)
  int64_t sum_p, sum_p2;
  double tol;
  int32_t max_sweeps;
  int32_t* flags;
  unsigned long long* stats;
};

template <class T, class V, int NT, int PMAX, int TI, int CI>
__global__ void __launch_bounds__(NT, 32768 / (NT * 32))
    k_fwd_persist_jt2(Prob<T, V> P, PersistArgs<T> a, int sched_off, int warm_start) {
  const int blk = P.psd_sched[sched_off + blockIdx.x];
  const int inst = P.row_inst[P.psd_row0[blk]];
  const int64_t c0 = P.col_off[inst], c1 = P.col_off[inst + 1];
  const int64_t r0 = P.row_off[inst], r1 = P.row_off[inst + 1];
  const int64_t n = P.n_total, m = P.m_total;
  for (int32_t k = a.k0; k < a.k1; ++k) {
    const int64_t slot = k - a.k0;
    const T* x = a.xs + slot * n;
    const T* s = a.ss + slot * m;
    const T* y = a.ys + slot * m;
    T* xn = a.xs + (slot + 1) * n;
    T* sn = a.ss + (slot + 1) * m;
    T* yn = a.ys + (slot + 1) * m;
    T* xt = a.xts + slot * n;
    T* st = a.sts + slot * m;
    const T* rho = a.rho + (int64_t)k * m;
    const T* alpha = a.alpha + (int64_t)k * P.ninst;
    const T* dinv = a.dinv + (int64_t)k * n;
    const double sigma = a.sigma[k];
    // a3 / a4: xi and x~ = D^-1 xi (as k_rhs for a diagonal instance)
    for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) {
      T acc = (T)sigma * x[j] - P.q[j];
      for (int64_t e = P.AT_rp[j]; e < P.AT_rp[j + 1]; ++e) {
        const int32_t r = P.AT_ci[e];
        acc += (T)ldv(P.AT_v, e) * (y[r] + rho[r] * (P.b[r] - s[r]));
      }
      xt[j] = acc * dinv[j];
    }
    __syncthreads();
    // a5, a6, a8 for the separable rows, s~ of every row, relaxed x (as k_post)
    const T al = alpha[inst];
    for (int64_t r = r0 + threadIdx.x; r < r1; r += NT) {
      T acc = T(0);
      for (int64_t e = P.A_rp[r]; e < P.A_rp[r + 1]; ++e) acc += (T)ldv(P.A_v, e) * xt[P.A_ci[e]];
      const T str = P.b[r] - acc;
      st[r] = str;
      const uint8_t kind = P.row_kind[r];
      if (kind <= K_BOX) {
        const T rh = rho[r];
        const T sh = al * str + (T(1) - al) * s[r];
        const T v = sh + y[r] / rh;
        T sp;
        if (kind == K_ZERO) sp = T(0);
        else if (kind == K_NONNEG) sp = v > T(0) ? v : T(0);
        else sp = fmin(fmax(v, P.box_l[r]), P.box_u[r]);
        const T ynr = y[r] + rh * (sh - sp);
        sn[r] = sp;
        yn[r] = ynr;
        if (!finite_(ynr) || !finite_(sp)) atomicOr(&a.flags[inst], F_NONFINITE);
      }
    }
    for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) xn[j] = al * xt[j] + (T(1) - al) * x[j];
    __syncthreads();
    // a7, a8: the PSD block, warm-started from the previous step's eigenvectors
    const T* U_prev = nullptr;
    if (warm_start && k > 0) U_prev = slot == 0 ? a.U_warm : a.Us + (slot - 1) * a.sum_p2;
    PsdIterIO<T> io{st, s, y, rho, alpha, sn, yn, P.row_inst};
    jt2_project<T, V, NT, PMAX, TI, CI>(P, io, a.lams + slot * a.sum_p, a.Us + slot * a.sum_p2, a.tol,
                                        a.max_sweeps, a.flags, blk, a.stats, U_prev);
    __syncthreads();
  }
}

}  // namespace cosmo
