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
#include "kernels_jt.cuh"

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

// round-robin pair k of round `rd` (0 <= rd < pe-1, 0 <= k < pe/2) for pe
// (even) indices; index pe-1 is fixed, the others rotate.  The sums stay in
// [0, 2m), so one conditional subtraction replaces the modulo.
__device__ __forceinline__ void rr_pair(int rd, int k, int pe, int& a, int& b) {
  const int m = pe - 1;
  if (k == 0) {
    a = m;
    b = rd;
  } else {
    a = rd + k;
    if (a >= m) a -= m;
    b = rd - k + m;
    if (b >= m) b -= m;
  }
}

template <class T> __device__ __forceinline__ T hypot_(T a, T b);
template <> __device__ __forceinline__ float hypot_(float a, float b) { return hypotf(a, b); }
template <> __device__ __forceinline__ double hypot_(double a, double b) { return hypot(a, b); }
template <class T> __device__ __forceinline__ T rsqrt_(T a);
template <> __device__ __forceinline__ float rsqrt_(float a) { return rsqrtf(a); }
template <> __device__ __forceinline__ double rsqrt_(double a) { return rsqrt(a); }

// One rotation of the round-robin schedule: pair (a, b) packed as a | b << 16
// and its (c, s), in one 16-byte record (two for double).
template <class T> struct __align__(16) PairRec { uint32_t ab; uint32_t pad; T c, s; };
template <> struct __align__(16) PairRec<float> { uint32_t ab; float c, s, pad; };

// Cyclic Jacobi on the symmetric matrix A (pe x ld, zero-padded; only the
// upper triangle is read and kept) in shared memory; V <- V J_1 J_2 ... (V
// starts as the identity, or holds a warm start).  Stops when off(A) <=
// tol' ||A||_F with tol' = max(tol, 4 eps sqrt(p)) (below that the rounding
// of the rotations themselves keeps off(A) from shrinking), or when from the
// fifth sweep on a sweep fails to halve off(A)^2 (quadratic convergence has
// ended at the rounding floor); returns the number of sweeps run, negative if
// max_sweeps was reached first.
//
// Rotations with |a_pq| <= tol' ||A||_F / (4p) are skipped: if every
// remaining coupling is that small, off(A) <= tol' ||A||_F / 4 already.  A
// round in which no pair rotates skips its updates.
//
// Rounds are software-pipelined.  Phase X: every thread applies round r's
// rotations to the 2x2 blocks (k, l), k <= l, of A's upper triangle (entry
// (r, c) at [min][max]), from a precomputed triangular index table.  Phase Y:
// the first warps compute round r+1's pairs and rotations from the updated A
// into the other half of a double buffer while the remaining warps apply round
// r's rotations to V, one warp per column pair, lanes over rows (odd stride
// ld: no bank conflicts).  Two barriers per round.
// Shared scratch: recs [2 pe/2] PairRec<T>, tri [np(np+1)/2] u32.
template <class T>
__device__ __forceinline__ bool jacobi_rotations(const T* A, PairRec<T>* rec, int rd, int p,
                                                 int pe, int ld, int first, int stride,
                                                 T thresh) {
  const int np = pe / 2;
  bool any = false;
  for (int k = first; k < np; k += stride) {
    int a, b;
    rr_pair(rd, k, pe, a, b);
    T c = T(1), s = T(0);
    if (a < p && b < p) {
      // only the upper triangle of A is kept
      const T apq = a < b ? A[a * ld + b] : A[b * ld + a];
      if (fabs(apq) > thresh) {
        // t = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = theta / phi, written
        // as sign(theta) phi / (|theta| + sqrt(theta^2 + phi^2)): one root and
        // one division; the rotation is skipped if the root under/overflows
        const T theta = A[b * ld + b] - A[a * ld + a];
        const T phi = T(2) * apq;
        const T r = sqrt(theta * theta + phi * phi);
        if (r > T(0) && r <= MaxVal<T>::v) {
          const T t = copysign(T(1), theta) * phi / (fabs(theta) + r);
          c = rsqrt_(T(1) + t * t);
          s = t * c;
          any = true;
        }
      }
    }
    PairRec<T> pr;
    pr.ab = (uint32_t)a | ((uint32_t)b << 16);
    pr.c = c;
    pr.s = s;
    rec[k] = pr;
  }
  return any;
}

template <class T>
__device__ int jacobi_eig(T* A, T* V, PairRec<T>* rec2, uint32_t* tri, double* red, int p,
                          double tol, int max_sweeps, bool v_identity = true) {
  const int pe = psd_pe(p), ld = psd_ld(p), np = pe / 2;
  const int ntri = np * (np + 1) / 2;
  const int nt = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = nt >> 5;
  // warps that compute rotations in phase Y; the rest update V meanwhile
  const int rot_warps = (np + 31) / 32;
  const bool split = nwarps >= rot_warps + 2;
  const int v_first_warp = split ? rot_warps : 0;
  const int v_warps = nwarps - v_first_warp;
  if (v_identity) {
    for (int e = threadIdx.x; e < pe * ld; e += nt) {
      const int i = e / ld, j = e % ld;
      V[e] = (i == j) ? T(1) : T(0);
    }
  }
  for (int e = threadIdx.x; e < ntri; e += nt) {
    int k, l;
    svec_ij(e, k, l);           // k <= l
    tri[e] = (uint32_t)k | ((uint32_t)l << 16);
  }
  __syncthreads();
  const double tol_eff = fmax(tol, 4.0 * Eps<T>::v * sqrt((double)p));
  const double tol2 = tol_eff * tol_eff;
  double prev_off2 = 0.0;
  int result = -max_sweeps;
  for (int sweep = 0;; ++sweep) {
    double acc[2] = {0.0, 0.0};   // off-diagonal and diagonal sums of squares (upper triangle)
    for (int e = threadIdx.x; e < p * (p + 1) / 2; e += nt) {
      int i, j;
      svec_ij(e, i, j);
      const double v = (double)A[i * ld + j];
      if (i == j) acc[1] += v * v;
      else acc[0] += v * v;
    }
    block_sum<2>(acc, red);
    const double off2 = 2.0 * acc[0], tot2 = off2 + acc[1];
    if (off2 <= tol2 * tot2 || (sweep >= 5 && off2 > 0.5 * prev_off2)) { result = sweep; break; }
    if (sweep >= max_sweeps) break;
    prev_off2 = off2;
    const T thresh = (T)(tol_eff * sqrt(tot2) / (4.0 * p));
    // __syncthreads_or hands every thread the OR: whether the round rotates
    bool active = __syncthreads_or(jacobi_rotations(A, rec2, 0, p, pe, ld, threadIdx.x, nt, thresh));
    for (int rd = 0; rd < pe - 1; ++rd) {
      const PairRec<T>* rec = rec2 + (rd & 1) * np;
      // ---- phase X: A <- J'AJ on the 2x2 blocks (k, l), k <= l, on the upper
      // triangle only; two blocks per thread in flight (all loads before any
      // store: blocks are disjoint)
      if (active) {
        for (int e0 = threadIdx.x; e0 < ntri; e0 += 2 * nt) {
          T x[2][4], cc[2][2], ss[2][2];
          int o[2][4];
          bool v[2], dg[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int e = e0 + u * nt;
            v[u] = e < ntri;
            const uint32_t kl = tri[v[u] ? e : 0];
            const int k = (int)(kl & 0xffffu), l = (int)(kl >> 16);
            dg[u] = k == l;
            const PairRec<T> rk = rec[k], rl = rec[l];
            const int ak = (int)(rk.ab & 0xffffu), bk = (int)(rk.ab >> 16);
            const int al = (int)(rl.ab & 0xffffu), bl = (int)(rl.ab >> 16);
            cc[u][0] = rk.c; ss[u][0] = rk.s;
            cc[u][1] = rl.c; ss[u][1] = rl.s;
            o[u][0] = ak < al ? ak * ld + al : al * ld + ak;
            o[u][1] = ak < bl ? ak * ld + bl : bl * ld + ak;
            o[u][2] = bk < al ? bk * ld + al : al * ld + bk;
            o[u][3] = bk < bl ? bk * ld + bl : bl * ld + bk;
            x[u][0] = A[o[u][0]];
            x[u][1] = A[o[u][1]];
            x[u][2] = A[o[u][2]];
            x[u][3] = A[o[u][3]];
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (!v[u]) continue;
            const T ck = cc[u][0], sk = ss[u][0], cl = cc[u][1], sl = ss[u][1];
            // rows: [r_a; r_b] <- [[c, -s], [s, c]] [r_a; r_b]
            const T y11 = ck * x[u][0] - sk * x[u][2], y12 = ck * x[u][1] - sk * x[u][3];
            const T y21 = sk * x[u][0] + ck * x[u][2], y22 = sk * x[u][1] + ck * x[u][3];
            // columns: [c_a, c_b] <- [c_a, c_b] [[c, s], [-s, c]]
            const T z11 = cl * y11 - sl * y12, z12 = sl * y11 + cl * y12;
            const T z21 = cl * y21 - sl * y22, z22 = sl * y21 + cl * y22;
            if (dg[u]) {
              // (a,a), (a,b)=(b,a), (b,b): the rotation annihilates the coupling
              A[o[u][0]] = z11;
              if (ck != T(1) || sk != T(0)) A[o[u][1]] = T(0);
              A[o[u][3]] = z22;
            } else {
              A[o[u][0]] = z11;
              A[o[u][1]] = z12;
              A[o[u][2]] = z21;
              A[o[u][3]] = z22;
            }
          }
        }
      }
      __syncthreads();
      // ---- phase Y: rotations of round rd+1 (first warps) || V <- V J_rd
      const bool more = rd + 1 < pe - 1;
      bool any_next = false;
      PairRec<T>* rec_next = rec2 + ((rd + 1) & 1) * np;
      if (split) {
        if (warp < rot_warps && more)
          any_next = jacobi_rotations(A, rec_next, rd + 1, p, pe, ld, threadIdx.x, rot_warps * 32, thresh);
      } else if (more) {
        any_next = jacobi_rotations(A, rec_next, rd + 1, p, pe, ld, threadIdx.x, nt, thresh);
      }
      if (active && warp >= v_first_warp) {
        // one warp per column pair l; lanes over rows (conflict-free)
        for (int l = warp - v_first_warp; l < np; l += v_warps) {
          const PairRec<T> rl = rec[l];
          if (rl.c == T(1) && rl.s == T(0)) continue;
          const int al = (int)(rl.ab & 0xffffu), bl = (int)(rl.ab >> 16);
          for (int i0 = lane; i0 < pe; i0 += 64) {
            T va[2], vb[2];
            const int i1 = i0 + 32;
            va[0] = V[i0 * ld + al];
            vb[0] = V[i0 * ld + bl];
            if (i1 < pe) { va[1] = V[i1 * ld + al]; vb[1] = V[i1 * ld + bl]; }
            V[i0 * ld + al] = rl.c * va[0] - rl.s * vb[0];
            V[i0 * ld + bl] = rl.s * va[0] + rl.c * vb[0];
            if (i1 < pe) {
              V[i1 * ld + al] = rl.c * va[1] - rl.s * vb[1];
              V[i1 * ld + bl] = rl.s * va[1] + rl.c * vb[1];
            }
          }
        }
      }
      active = __syncthreads_or(any_next);
    }
  }
  return result;
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

// Conflict-free variant: lane (threadIdx.x % 32) owns columns j = lane + 32 b,
// warp w owns rows i = w + TY a (TY warps): B(k, j) loads are consecutive
// across lanes (or stride ld, odd) and A(i, k) loads are warp broadcasts.
template <class T, int TM, int TN, class F>
__device__ __forceinline__ void smem_gemm_w(int p, const T* A, int ar, int ac, const T* B, int br,
                                            int bc, F f) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, TY = blockDim.x >> 5;
  for (int i0 = w; i0 < p; i0 += TM * TY) {
    for (int j0 = lane; j0 < p; j0 += TN * 32) {
      T acc[TM][TN];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = T(0);
      int ii[TM], jj[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) ii[a] = min(i0 + a * TY, p - 1);
#pragma unroll
      for (int b = 0; b < TN; ++b) jj[b] = min(j0 + b * 32, p - 1);
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
          if (i0 + a * TY < p && j0 + b * 32 < p) f(i0 + a * TY, j0 + b * 32, acc[a][b]);
    }
  }
}

// tile shape by CTA size: 128 threads (blocks up to 32) 8x1, 256 (up to 56)
// 7x2, 512 (larger) 5x3 outputs per thread
template <class T, class F>
__device__ __forceinline__ void smem_gemm_auto(int p, const T* A, int ar, int ac, const T* B,
                                               int br, int bc, F f) {
  if (blockDim.x >= 512) smem_gemm_w<T, 5, 3>(p, A, ar, ac, B, br, bc, f);
  else if (blockDim.x >= 256) smem_gemm_w<T, 7, 2>(p, A, ar, ac, B, br, bc, f);
  else smem_gemm_w<T, 8, 1>(p, A, ar, ac, B, br, bc, f);
}

// shared memory the Jacobi projection needs for order p (bytes)
// layout: A, V [pe x ld] T | recs [pe] PairRec<T> (16-aligned) | sel [pe + 2]
// int | flags [4] int | tri [np(np+1)/2] u32 | red (8-aligned) [2 nt/32] double
template <class T>
__host__ __device__ inline size_t psd_fwd_smem(int p, int nt) {
  const int pe = psd_pe(p), ld = psd_ld(p), np = pe / 2;
  return (size_t)2 * pe * ld * sizeof(T) + 16 + (size_t)pe * sizeof(PairRec<T>) +
         (size_t)(pe + 6) * sizeof(int) + (size_t)(np * (np + 1) / 2) * sizeof(uint32_t) +
         (size_t)(2 * (nt / 32)) * sizeof(double) + 64;
}

// with a warm start a third pe x ld buffer W follows the red array
template <class T>
__host__ __device__ inline size_t psd_fwd_smem_warm(int p, int nt) {
  const int pe = psd_pe(p), ld = psd_ld(p);
  return psd_fwd_smem<T>(p, nt) + (size_t)pe * ld * sizeof(T) + 16;
}

template <class T>
struct JacobiSmem {
  T* A; T* V; PairRec<T>* rec; int* sel; int* flag2; uint32_t* tri; double* red;
  __device__ JacobiSmem(unsigned char* raw, int p) {
    const int pe = psd_pe(p), ld = psd_ld(p), np = pe / 2;
    A = reinterpret_cast<T*>(raw);
    V = A + pe * ld;
    rec = reinterpret_cast<PairRec<T>*>((reinterpret_cast<uintptr_t>(V + pe * ld) + 15) & ~uintptr_t(15));
    sel = reinterpret_cast<int*>(rec + 2 * np);
    flag2 = sel + pe + 2;
    tri = reinterpret_cast<uint32_t*>(flag2 + 4);
    red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(tri + np * (np + 1) / 2) + 7) & ~uintptr_t(7));
  }
  // third buffer, only valid when the launch sized shared memory with psd_fwd_smem_warm
  __device__ T* W(int nt) const {
    return reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(red + 2 * (nt / 32)) + 15) & ~uintptr_t(15));
  }
};
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
                                                int32_t* flags, int sched_off,
                                                unsigned long long* stats, const T* U_prev) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = P.psd_sched[sched_off + blockIdx.x];
  const int p = P.psd_p[blk];
  const int pe = psd_pe(p), ld = psd_ld(p);
  const int64_t row0 = P.psd_row0[blk];
  JacobiSmem<T> sm(smraw, p);
  T* A = sm.A;
  T* Vm = sm.V;
  int* sel = sm.sel;
  const int inst = io.row_inst[row0];
  const T al = io.alpha[inst], rh = io.rho[row0];
  const int d = p * (p + 1) / 2;
  const bool warm = U_prev != nullptr;
  if (warm) {
    // previous step's eigenvectors (column-major) into V, then one
    // Newton-Schulz step V <- 1.5 V - 0.5 V (V'V) to restore orthogonality
    T* W = sm.W(NT);
    const T* Up = U_prev + P.psd_uoff[blk];
    for (int e = threadIdx.x; e < pe * ld; e += NT) { Vm[e] = T(0); A[e] = T(0); W[e] = T(0); }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += NT) {
      const int k = e / p, i = e - k * p;
      Vm[i * ld + k] = Up[e];
    }
    if (threadIdx.x == 0 && (p & 1)) Vm[p * ld + p] = T(1);  // padding index
    __syncthreads();
    smem_gemm_auto<T>(p, Vm, 1, ld, Vm, ld, 1, [&](int i, int j, T v) { W[i * ld + j] = v; });
    __syncthreads();
    smem_gemm_auto<T>(p, Vm, ld, 1, W, ld, 1, [&](int i, int j, T v) { A[i * ld + j] = v; });
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += NT) {
      const int i = e / p, j = e - i * p;
      Vm[i * ld + j] = T(1.5) * Vm[i * ld + j] - T(0.5) * A[i * ld + j];
    }
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < pe * ld; e += NT) A[e] = T(0);
    __syncthreads();
  }
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
  if (warm) {
    // B = V' S V, nearly diagonal when the iterate moved little
    T* W = sm.W(NT);
    smem_gemm_auto<T>(p, A, ld, 1, Vm, ld, 1, [&](int i, int j, T v) { W[i * ld + j] = v; });
    __syncthreads();
    smem_gemm_auto<T>(p, Vm, 1, ld, W, ld, 1, [&](int i, int j, T v) { A[i * ld + j] = v; });
    __syncthreads();
  }
  const int sweeps = jacobi_eig(A, Vm, sm.rec, sm.tri, sm.red, p, tol, max_sweeps, !warm);
  if (threadIdx.x == 0) {
    if (sweeps < 0) atomicOr(&flags[inst], F_EIG_CAP);
    if (stats) {
      atomicAdd(&stats[0], (unsigned long long)(sweeps < 0 ? -sweeps : sweeps));
      atomicAdd(&stats[1], 1ull);
    }
  }
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

// a7 with the slot-layout Jacobi solver of kernels_jt.cuh: the same
// projection, relaxation input and fused dual update as k_psd_fwd; the
// eigenvectors are kept by row (Vt), the warm start's products are formed in
// that layout, and the solver works on 2x2 tiles with one barrier per round.
// 64 registers per thread at most, so that two CTAs of 512 threads (or a
// 512- and a 256-thread CTA of different size classes) share an SM
template <class T, class V, int NT, int IPT>
__global__ void __launch_bounds__(NT, 32768 / (NT * 32)) k_psd_fwd_jt(Prob<T, V> P, PsdIterIO<T> io, T* lam_slot,
                                                   T* U_slot, double tol, int max_sweeps,
                                                   int32_t* flags, int sched_off,
                                                   unsigned long long* stats, const T* U_prev) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = P.psd_sched[sched_off + blockIdx.x];
  const int p = P.psd_p[blk];
  const int pe = psd_pe(p), np = pe / 2, ldv = jt_ldv(p), lds = jt_lds(p), ntri = jt_ntri(p);
  const int64_t row0 = P.psd_row0[blk];
  JtSmem<T> sm(smraw, p);
  T* Vt = sm.Vt;
  T* S = sm.S;
  T* X = sm.X;
  const int inst = io.row_inst[row0];
  const T al = io.alpha[inst], rh = io.rho[row0];
  const int d = p * (p + 1) / 2;
  const bool warm = U_prev != nullptr;
  for (int e = threadIdx.x; e < pe * ldv; e += NT) {
    const int i = e / ldv, j = e - i * ldv;
    Vt[e] = (!warm && i == j && i < p) ? T(1) : T(0);
  }
  __syncthreads();
  if (warm) {
    // previous step's eigenvectors as rows (orthogonal to rounding: every
    // step hands over re-orthogonalised vectors, see below)
    const T* Up = U_prev + P.psd_uoff[blk];
    for (int e = threadIdx.x; e < p * p; e += NT) {
      const int j = e / p, i = e - j * p;
      Vt[j * ldv + i] = Up[e];
    }
  }
  // S = smat(v), v = alpha s~ + (1 - alpha) s + y / rho
  auto load_S = [&]() {
    for (int e = threadIdx.x; e < d; e += NT) {
      int i, j;
      svec_ij(e, i, j);
      const int64_t r = row0 + e;
      T v = al * io.st[r] + (T(1) - al) * io.s[r] + io.y[r] / rh;
      if (i != j) v *= (T)kInvSqrt2;
      S[i * lds + j] = v;
      S[j * lds + i] = v;
    }
  };
  load_S();
  __syncthreads();
  if (warm) {
    // B = V' S V (upper triangle read below), nearly diagonal when the
    // iterate moved little: C = Vt S into X, then C Vt' into S
    smem_gemm_auto<T>(p, Vt, ldv, 1, S, lds, 1, [&](int i, int j, T v) { X[i * lds + j] = v; });
    __syncthreads();
    smem_gemm_auto<T>(p, X, lds, 1, Vt, 1, ldv, [&](int i, int j, T v) { S[i * lds + j] = v; });
    __syncthreads();
  }
  // tiles of round 0 (slot layout, four planes of ntri values) from the upper triangle of S
  T* tb0 = X;
  T* tb1 = X + 4 * ntri;
  for (int e = threadIdx.x; e < ntri; e += NT) {
    int k, l;
    svec_ij(e, k, l);
    const int a0 = jt_slot_index(0, 2 * k, np), a1 = jt_slot_index(0, 2 * k + 1, np);
    const int b0 = jt_slot_index(0, 2 * l, np), b1 = jt_slot_index(0, 2 * l + 1, np);
    auto at = [&](int i, int j) -> T {
      if (i >= p || j >= p) return T(0);
      return i <= j ? S[i * lds + j] : S[j * lds + i];
    };
    tb0[e] = at(a0, b0);
    tb0[ntri + e] = at(a0, b1);
    tb0[2 * ntri + e] = at(a1, b0);
    tb0[3 * ntri + e] = at(a1, b1);
  }
  __syncthreads();
  auto off = [&](const void* q) { return (uint32_t)(reinterpret_cast<uintptr_t>(q) - reinterpret_cast<uintptr_t>(smraw)); };
  uint32_t fin_off = off(tb0);
  const int sweeps = jt_solve<T, NT, IPT>(smraw, off(tb0), off(tb1), off(Vt), off(sm.rec), sm.red, p, tol,
                                          max_sweeps, &fin_off);
  const T* fin = reinterpret_cast<const T*>(smraw + fin_off);
  if (threadIdx.x == 0) {
    if (sweeps < 0) atomicOr(&flags[inst], F_EIG_CAP);
    if (stats) {
      atomicAdd(&stats[0], (unsigned long long)(sweeps < 0 ? -sweeps : sweeps));
      atomicAdd(&stats[1], 1ull);
    }
  }
  (void)fin;   // the refinement below starts again from S and the rotated basis
  // Refinement.  In FP32 the accumulated rotations leave Vt orthogonal only to
  // about sqrt(#rotations) * eps (a few 1e-6 over a cold solve), which alone
  // would put a few 1e-6 of relative error in the projection and in the
  // Daleckii-Krein backward.  So (1) one Newton-Schulz step Vt <- 1.5 Vt -
  // 0.5 (Vt Vt') Vt restores orthogonality to rounding; (2) a Rayleigh-Ritz
  // step in that basis, A = Vt S Vt' (S formed again from the iterate), gives
  // the eigenvalues as its diagonal L and leaves its off-diagonal E, of the
  // size of the solver's stopping tolerance; (3) Pi(S) = Vt' (max(L, 0) +
  // G o E) Vt (Eq. psd-proj), where G is the Loewner matrix of max(x, 0) at L
  // (Eq. lowner: the Daleckii-Krein derivative the backward applies), which
  // removes the O(||E||) error of dropping E.  G of two same-sign eigenvalues
  // is 1 or 0 without a division, and of mixed signs l+ / (l+ - l-) (no
  // cancellation).
  smem_gemm_auto<T>(p, Vt, ldv, 1, Vt, 1, ldv, [&](int i, int j, T v) { X[i * lds + j] = v; });
  __syncthreads();
  smem_gemm_auto<T>(p, X, lds, 1, Vt, ldv, 1, [&](int i, int j, T v) { S[i * lds + j] = v; });
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += NT) {
    const int i = e / p, j = e - i * p;
    Vt[i * ldv + j] = T(1.5) * Vt[i * ldv + j] - T(0.5) * S[i * lds + j];
  }
  __syncthreads();
  load_S();
  __syncthreads();
  smem_gemm_auto<T>(p, Vt, ldv, 1, S, lds, 1, [&](int i, int j, T v) { X[i * lds + j] = v; });
  __syncthreads();
  // X = Vt S: eigenvalues, the tape, the selected index set, then Pi from the
  // rows of the Rayleigh-Ritz matrix at that set (the routine of
  // kernels_jt.cuh that k_psd_fwd_jt2 runs too: both give the same bits)
  T* lamv = sm.lamv;
  int* const sel = sm.sel;
  jt_rr_diag<T>(p, Vt, ldv, X, lds, lamv);
  __syncthreads();
  jt_select<T>(p, lamv, sel, p);
  T* lam = lam_slot + P.psd_loff[blk];
  T* U = U_slot + P.psd_uoff[blk];
  for (int k = threadIdx.x; k < p; k += NT) lam[k] = lamv[k];
  for (int e = threadIdx.x; e < p * p; e += NT) {
    const int k = e / p, i = e - k * p;
    U[e] = Vt[k * ldv + i];
  }
  __syncthreads();
  const int ns = sel[p];
  const bool usepos = sel[p + 1] != 0;
  jt_lowrank_rows<T>(p, Vt, ldv, X, lds, S, lds, lamv, sel, ns, usepos);
  __syncthreads();
  jt_lowrank_wz<T>(p, Vt, ldv, X, lds, S, lds, lamv, ns, usepos);
  __syncthreads();
  for (int e = threadIdx.x; e < d; e += NT) {
    int i, j;
    svec_ij(e, i, j);
    const int64_t r = row0 + e;
    const T sh = al * io.st[r] + (T(1) - al) * io.s[r];
    T sij = sh + io.y[r] / rh;                       // S(i, j) (svec entry scaled back)
    if (i != j) sij *= (T)kInvSqrt2;
    T out = jt_lowrank_entry<T>(i, j, Vt, ldv, X, lds, sel, ns, usepos, sij);
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
                                                const T* U_slot, double dk_tau_rel, int sched_off) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = P.psd_sched[sched_off + blockIdx.x];
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
  JacobiSmem<T> sm(smraw, p);
  T* A = sm.A;
  T* Vm = sm.V;
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
  const int sweeps = jacobi_eig(A, Vm, sm.rec, sm.tri, sm.red, p, tol, max_sweeps);
  if (sweeps < 0 && threadIdx.x == 0 && flag) atomicOr(flag, F_EIG_CAP);
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
