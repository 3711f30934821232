// PSD-cone kernels: projection Pi(S) = U max(Lambda, 0) U' (Sec. 2.4,
// Eq. psd-proj) via a cyclic Jacobi eigensolver, and the Daleckii-Krein
// backward S_bar = U (L o (U' T_bar U)) U' (Eqs. psd-cotangent-dk, lowner).
//
// One CTA per PSD block; the block lives in shared memory for its whole
// life.  Jacobi uses the round-robin ("tournament") parallel ordering
// (Brent & Luk 1985): in each of the pe-1 rounds of a sweep the pe/2 index
// pairs are disjoint, so the two-sided update J'AJ splits into independent
// 2x2 blocks that threads update in one pass.  Rotation angles follow the
// symmetric 2x2 Schur decomposition (Golub & Van Loan, Alg. 8.5.1).
#pragma once

#include "common.cuh"

namespace cosmo {

constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kInvSqrt2 = 0.70710678118654752440;

__host__ __device__ __forceinline__ int psd_pe(int p) { return p + (p & 1); }
__host__ __device__ __forceinline__ int psd_ld(int p) { return psd_pe(p) + 1; }

// svec position e -> (i, j), i <= j, column-major upper triangle
__device__ __forceinline__ void svec_ij(int e, int& i, int& j) {
  int jj = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((jj + 1) * (jj + 2) / 2 <= e) ++jj;
  while (jj * (jj + 1) / 2 > e) --jj;
  j = jj;
  i = e - jj * (jj + 1) / 2;
}

// round-robin pair k of round `rd` for pe (even) indices; index pe-1 is fixed
__device__ __forceinline__ void rr_pair(int rd, int k, int pe, int& a, int& b) {
  const int m = pe - 1;
  if (k == 0) {
    a = m;
    b = rd % m;
  } else {
    a = (rd + k) % m;
    b = (rd - k + m) % m;
  }
}

template <class T> __device__ __forceinline__ T hypot_(T a, T b);
template <> __device__ __forceinline__ float hypot_(float a, float b) { return hypotf(a, b); }
template <> __device__ __forceinline__ double hypot_(double a, double b) { return hypot(a, b); }
template <class T> __device__ __forceinline__ T rsqrt_(T a);
template <> __device__ __forceinline__ float rsqrt_(float a) { return rsqrtf(a); }
template <> __device__ __forceinline__ double rsqrt_(double a) { return rsqrt(a); }

// Cyclic Jacobi on the symmetric matrix A (pe x ld, zero-padded) in shared
// memory; V <- accumulated rotations (starts as the identity).  Stops when
// off(A) <= tol ||A||_F or after max_sweeps (returns false then).
template <class T>
__device__ bool jacobi_eig(T* A, T* V, T* cs, double* red, int p, double tol, int max_sweeps) {
  const int pe = psd_pe(p), ld = psd_ld(p), np = pe / 2;
  for (int e = threadIdx.x; e < pe * ld; e += blockDim.x) {
    const int i = e / ld, j = e % ld;
    V[e] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  const double tol2 = tol * tol;
  bool ok = false;
  for (int sweep = 0;; ++sweep) {
    double acc[2] = {0.0, 0.0};
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      const int i = e / p, j = e % p;
      const double v = (double)A[i * ld + j];
      acc[1] += v * v;
      if (i != j) acc[0] += v * v;
    }
    block_sum<2>(acc, red);
    if (acc[0] <= tol2 * acc[1]) { ok = true; break; }
    if (sweep >= max_sweeps) break;
    for (int rd = 0; rd < pe - 1; ++rd) {
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        int a, b;
        rr_pair(rd, k, pe, a, b);
        T c = T(1), s = T(0);
        if (a < p && b < p) {
          const T apq = A[a * ld + b];
          if (apq != T(0)) {
            const T tau = (A[b * ld + b] - A[a * ld + a]) / (T(2) * apq);
            const T t = copysign(T(1), tau) / (fabs(tau) + hypot_(T(1), tau));
            c = rsqrt_(T(1) + t * t);
            s = t * c;
          }
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // A <- J'AJ as independent 2x2 blocks (pair k rows, pair l columns)
      for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
        const int k = e / np, l = e % np;
        int ak, bk, al, bl;
        rr_pair(rd, k, pe, ak, bk);
        rr_pair(rd, l, pe, al, bl);
        const T ck = cs[2 * k], sk = cs[2 * k + 1], cl = cs[2 * l], sl = cs[2 * l + 1];
        const T x11 = A[ak * ld + al], x12 = A[ak * ld + bl];
        const T x21 = A[bk * ld + al], x22 = A[bk * ld + bl];
        // rows: [r_a; r_b] <- [[c, -s], [s, c]] [r_a; r_b]
        const T y11 = ck * x11 - sk * x21, y12 = ck * x12 - sk * x22;
        const T y21 = sk * x11 + ck * x21, y22 = sk * x12 + ck * x22;
        // columns: [c_a, c_b] <- [c_a, c_b] [[c, s], [-s, c]]
        T z11 = cl * y11 - sl * y12, z12 = sl * y11 + cl * y12;
        T z21 = cl * y21 - sl * y22, z22 = sl * y21 + cl * y22;
        if (k == l) { z12 = T(0); z21 = T(0); }
        A[ak * ld + al] = z11; A[ak * ld + bl] = z12;
        A[bk * ld + al] = z21; A[bk * ld + bl] = z22;
      }
      // V <- V J (rows i, pair l)
      for (int e = threadIdx.x; e < pe * np; e += blockDim.x) {
        const int i = e / np, l = e % np;
        int al, bl;
        rr_pair(rd, l, pe, al, bl);
        const T cl = cs[2 * l], sl = cs[2 * l + 1];
        const T va = V[i * ld + al], vb = V[i * ld + bl];
        V[i * ld + al] = cl * va - sl * vb;
        V[i * ld + bl] = sl * va + cl * vb;
      }
      __syncthreads();
    }
  }
  return ok;
}

// C(i, j) = sum_k A(i, k) B(k, j) for i, j < p, with A(i, k) = A[i*ar + k*ac],
// B(k, j) = B[k*br + j*bc]; each thread owns TM x TN outputs.  Epilogue f(i,
// j, value) stores the result.
template <class T, int TM, int TN, class F>
__device__ __forceinline__ void smem_gemm(int p, const T* A, int ar, int ac, const T* B, int br,
                                          int bc, F f) {
  const int nti = (p + TM - 1) / TM, ntj = (p + TN - 1) / TN;
  for (int t = threadIdx.x; t < nti * ntj; t += blockDim.x) {
    const int i0 = (t / ntj) * TM, j0 = (t % ntj) * TN;
    T acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) acc[a][b] = T(0);
    int ii[TM], jj[TN];
#pragma unroll
    for (int a = 0; a < TM; ++a) ii[a] = min(i0 + a, p - 1);
#pragma unroll
    for (int b = 0; b < TN; ++b) jj[b] = min(j0 + b, p - 1);
    for (int k = 0; k < p; ++k) {
      T av[TM], bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = A[ii[a] * ar + k * ac];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = B[k * br + jj[b] * bc];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b)
        if (i0 + a < p && j0 + b < p) f(i0 + a, j0 + b, acc[a][b]);
  }
}

template <class T, class F>
__device__ __forceinline__ void smem_gemm_auto(int p, const T* A, int ar, int ac, const T* B,
                                               int br, int bc, F f) {
  if (p >= 40) smem_gemm<T, 4, 4>(p, A, ar, ac, B, br, bc, f);
  else smem_gemm<T, 2, 2>(p, A, ar, ac, B, br, bc, f);
}

// shared memory the Jacobi projection needs for order p (bytes)
template <class T>
__host__ __device__ inline size_t psd_fwd_smem(int p, int nt) {
  const int pe = psd_pe(p), ld = psd_ld(p);
  return (size_t)2 * pe * ld * sizeof(T) + (size_t)pe * sizeof(T) + (size_t)pe * sizeof(int) +
         (size_t)(2 * (nt / 32)) * sizeof(double) + 64;
}
template <class T>
__host__ __device__ inline size_t psd_bwd_smem(int p, int nt) {
  const int pe = psd_pe(p), ld = psd_ld(p);
  return (size_t)3 * pe * ld * sizeof(T) + (size_t)pe * sizeof(double) +
         (size_t)(2 * (nt / 32)) * sizeof(double) + 64;
}

// Source/sink of one block's svec data for the projection kernel.
template <class T>
struct PsdIterIO {   // inside the unrolled iteration
  const T* st; const T* s; const T* y; const T* rho; const T* alpha;
  T* sn; T* yn;
  const int32_t* row_inst;
};

// a7: PSD projection inside iteration k, fused with the relaxation (the
// projection input v = alpha s~ + (1-alpha) s + y/rho) and the dual update.
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_psd_fwd(Prob<T, V> P, PsdIterIO<T> io, T* lam_slot,
                                                T* U_slot, double tol, int max_sweeps,
                                                int32_t* flags) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = P.psd_sched[blockIdx.x];
  const int p = P.psd_p[blk];
  const int pe = psd_pe(p), ld = psd_ld(p);
  const int64_t row0 = P.psd_row0[blk];
  T* A = reinterpret_cast<T*>(smraw);
  T* Vm = A + pe * ld;
  T* cs = Vm + pe * ld;
  int* sel = reinterpret_cast<int*>(cs + pe);
  double* red = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(sel + pe + 2) & ~uintptr_t(7));
  red = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(red) + 8);
  const int inst = io.row_inst[row0];
  const T al = io.alpha[inst], rh = io.rho[row0];
  const int d = p * (p + 1) / 2;
  for (int e = threadIdx.x; e < pe * ld; e += NT) A[e] = T(0);
  __syncthreads();
  for (int e = threadIdx.x; e < d; e += NT) {
    int i, j;
    svec_ij(e, i, j);
    const int64_t r = row0 + e;
    T v = al * io.st[r] + (T(1) - al) * io.s[r] + io.y[r] / rh;
    if (i != j) v *= (T)kInvSqrt2;
    A[i * ld + j] = v;
    A[j * ld + i] = v;
  }
  __syncthreads();
  const bool ok = jacobi_eig(A, Vm, cs, red, p, tol, max_sweeps);
  if (!ok && threadIdx.x == 0) atomicOr(&flags[inst], F_EIG_CAP);
  // tape: eigenvalues and eigenvectors (column-major per block)
  T* lam = lam_slot + P.psd_loff[blk];
  T* U = U_slot + P.psd_uoff[blk];
  for (int k = threadIdx.x; k < p; k += NT) lam[k] = A[k * ld + k];
  for (int e = threadIdx.x; e < p * p; e += NT) {
    const int k = e / p, i = e % p;
    U[e] = Vm[i * ld + k];
  }
  // reconstruction from the smaller of the positive / non-positive sets
  if (threadIdx.x == 0) {
    int npos = 0;
    for (int k = 0; k < p; ++k) npos += A[k * ld + k] > T(0);
    const bool usepos = npos <= p - npos;
    int c = 0;
    for (int k = 0; k < p; ++k)
      if ((A[k * ld + k] > T(0)) == usepos) sel[c++] = k;
    sel[pe] = c;
    sel[pe + 1] = usepos;
  }
  __syncthreads();
  const int nsel = sel[pe];
  const bool usepos = sel[pe + 1] != 0;
  for (int e = threadIdx.x; e < d; e += NT) {
    int i, j;
    svec_ij(e, i, j);
    T acc = T(0);
    for (int q = 0; q < nsel; ++q) {
      const int k = sel[q];
      acc += A[k * ld + k] * Vm[i * ld + k] * Vm[j * ld + k];
    }
    const int64_t r = row0 + e;
    const T sh = al * io.st[r] + (T(1) - al) * io.s[r];
    T out;
    if (usepos) {
      out = acc;
    } else {
      T sij = sh + io.y[r] / rh;            // svec entry of S
      if (i != j) sij *= (T)kInvSqrt2;
      out = sij - acc;
    }
    if (i != j) out *= (T)kSqrt2;
    const T yn = io.y[r] + rh * (sh - out);
    io.sn[r] = out;
    io.yn[r] = yn;
    if (!finite_(yn)) atomicOr(&flags[inst], F_NONFINITE);
  }
}

// Loewner matrix entry of f(x) = max(x, 0) (Eq. lowner): divided difference,
// or f'((li+lj)/2) with f'(0) = 1/2 when |li - lj| <= tau.  Double precision.
__device__ __forceinline__ double loewner_relu(double li, double lj, double tau) {
  if (fabs(li - lj) <= tau) {
    const double m = 0.5 * (li + lj);
    return m > 0.0 ? 1.0 : (m < 0.0 ? 0.0 : 0.5);
  }
  return (fmax(li, 0.0) - fmax(lj, 0.0)) / (li - lj);
}

// Daleckii-Krein core on one block in shared memory: G holds smat(g) on
// entry; U (row i, column k) the eigenvectors; lam the eigenvalues (double).
// On exit W holds U (L o (U'GU)), so S_bar(i, j) = sum_l W(i, l) U(j, l).
template <class T>
__device__ void dk_core(int p, T* Us, T* G, T* W, const double* lamd, double tau) {
  const int ld = psd_ld(p);
  // W = U' G
  smem_gemm_auto<T>(p, Us, 1, ld, G, ld, 1, [&](int k, int j, T v) { W[k * ld + j] = v; });
  __syncthreads();
  // G = (W U) o L
  smem_gemm_auto<T>(p, W, ld, 1, Us, ld, 1, [&](int k, int l, T v) {
    G[k * ld + l] = (T)((double)v * loewner_relu(lamd[k], lamd[l], tau));
  });
  __syncthreads();
  // W = U G
  smem_gemm_auto<T>(p, Us, ld, 1, G, ld, 1, [&](int i, int l, T v) { W[i * ld + l] = v; });
  __syncthreads();
}

template <class T>
struct PsdBwdIO {
  const T* g;     // cotangent at the projection output, svec rows (gproj)
  T* vbar;        // out, svec rows
  const int32_t* row_inst;
};

// b3 (PSD): vbar = svec(U (L o (U' smat(g) U)) U') per block
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_psd_bwd(Prob<T, V> P, PsdBwdIO<T> io, const T* lam_slot,
                                                const T* U_slot, double dk_tau_rel) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = P.psd_sched[blockIdx.x];
  const int p = P.psd_p[blk];
  const int pe = psd_pe(p), ld = psd_ld(p);
  const int64_t row0 = P.psd_row0[blk];
  T* Us = reinterpret_cast<T*>(smraw);
  T* G = Us + pe * ld;
  T* W = G + pe * ld;
  double* lamd = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(W + pe * ld + 1) & ~uintptr_t(7));
  lamd += 1;
  double* red = lamd + pe;
  const T* lam = lam_slot + P.psd_loff[blk];
  const T* U = U_slot + P.psd_uoff[blk];
  const int d = p * (p + 1) / 2;
  for (int e = threadIdx.x; e < p * p; e += NT) {
    const int k = e / p, i = e % p;
    Us[i * ld + k] = U[e];
  }
  for (int k = threadIdx.x; k < p; k += NT) lamd[k] = (double)lam[k];
  for (int e = threadIdx.x; e < d; e += NT) {
    int i, j;
    svec_ij(e, i, j);
    T v = io.g[row0 + e];
    if (i != j) v *= (T)kInvSqrt2;
    G[i * ld + j] = v;
    G[j * ld + i] = v;
  }
  __syncthreads();
  // max |lambda| of the block by one thread (p is at most a few hundred)
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < p; ++k) m = fmax(m, fabs(lamd[k]));
    red[0] = m;
  }
  __syncthreads();
  const double tau = dk_tau_rel * fmax(1.0, red[0]);
  dk_core<T>(p, Us, G, W, lamd, tau);
  for (int e = threadIdx.x; e < d; e += NT) {
    int i, j;
    svec_ij(e, i, j);
    T acc = T(0);
    for (int l = 0; l < p; ++l) acc = fma(W[i * ld + l], Us[j * ld + l], acc);
    if (i != j) acc *= (T)kSqrt2;
    io.vbar[row0 + e] = acc;
  }
}

// ---------------------------------------------------------------------------
// standalone batched projection / DK (no iterate): block j at svec offset
// off[j], eigen outputs at loff[j] / uoff[j]
// ---------------------------------------------------------------------------
template <class T>
struct PsdBatch {
  int32_t nblk;
  const int32_t* p; const int64_t* off; const int64_t* loff; const int64_t* uoff;
};

template <class T, int NT>
__global__ void __launch_bounds__(NT) k_psd_project_batch(PsdBatch<T> B, const T* v, T* out,
                                                          T* lam_out, T* U_out, double tol,
                                                          int max_sweeps, int32_t* flag) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = blockIdx.x;
  const int p = B.p[blk];
  const int pe = psd_pe(p), ld = psd_ld(p);
  T* A = reinterpret_cast<T*>(smraw);
  T* Vm = A + pe * ld;
  T* cs = Vm + pe * ld;
  int* sel = reinterpret_cast<int*>(cs + pe);
  double* red = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(sel + pe + 2) & ~uintptr_t(7));
  red = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(red) + 8);
  const int64_t o = B.off[blk];
  const int d = p * (p + 1) / 2;
  for (int e = threadIdx.x; e < pe * ld; e += NT) A[e] = T(0);
  __syncthreads();
  for (int e = threadIdx.x; e < d; e += NT) {
    int i, j;
    svec_ij(e, i, j);
    T x = v[o + e];
    if (i != j) x *= (T)kInvSqrt2;
    A[i * ld + j] = x;
    A[j * ld + i] = x;
  }
  __syncthreads();
  const bool ok = jacobi_eig(A, Vm, cs, red, p, tol, max_sweeps);
  if (!ok && threadIdx.x == 0 && flag) atomicOr(flag, F_EIG_CAP);
  if (lam_out)
    for (int k = threadIdx.x; k < p; k += NT) lam_out[B.loff[blk] + k] = A[k * ld + k];
  if (U_out)
    for (int e = threadIdx.x; e < p * p; e += NT) U_out[B.uoff[blk] + e] = Vm[(e % p) * ld + e / p];
  for (int e = threadIdx.x; e < d; e += NT) {
    int i, j;
    svec_ij(e, i, j);
    T acc = T(0);
    for (int k = 0; k < p; ++k) {
      const T l = A[k * ld + k];
      if (l > T(0)) acc += l * Vm[i * ld + k] * Vm[j * ld + k];
    }
    if (i != j) acc *= (T)kSqrt2;
    out[o + e] = acc;
  }
}

template <class T, int NT>
__global__ void __launch_bounds__(NT) k_psd_dk_batch(PsdBatch<T> B, const T* lam_in,
                                                     const T* U_in, const T* g, T* out,
                                                     double dk_tau_rel) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = blockIdx.x;
  const int p = B.p[blk];
  const int pe = psd_pe(p), ld = psd_ld(p);
  T* Us = reinterpret_cast<T*>(smraw);
  T* G = Us + pe * ld;
  T* W = G + pe * ld;
  double* lamd = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(W + pe * ld + 1) & ~uintptr_t(7));
  lamd += 1;
  double* red = lamd + pe;
  const int64_t o = B.off[blk];
  const T* lam = lam_in + B.loff[blk];
  const T* U = U_in + B.uoff[blk];
  const int d = p * (p + 1) / 2;
  for (int e = threadIdx.x; e < p * p; e += NT) Us[(e % p) * ld + e / p] = U[e];
  for (int k = threadIdx.x; k < p; k += NT) lamd[k] = (double)lam[k];
  for (int e = threadIdx.x; e < d; e += NT) {
    int i, j;
    svec_ij(e, i, j);
    T v = g[o + e];
    if (i != j) v *= (T)kInvSqrt2;
    G[i * ld + j] = v;
    G[j * ld + i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < p; ++k) m = fmax(m, fabs(lamd[k]));
    red[0] = m;
  }
  __syncthreads();
  const double tau = dk_tau_rel * fmax(1.0, red[0]);
  dk_core<T>(p, Us, G, W, lamd, tau);
  for (int e = threadIdx.x; e < d; e += NT) {
    int i, j;
    svec_ij(e, i, j);
    T acc = T(0);
    for (int l = 0; l < p; ++l) acc = fma(W[i * ld + l], Us[j * ld + l], acc);
    if (i != j) acc *= (T)kSqrt2;
    out[o + e] = acc;
  }
}

}  // namespace cosmo
