// PSD projection for blocks above the Jacobi cutoff: Householder
// tridiagonalisation (Golub & Van Loan, Alg. 8.3.1), explicit formation of Q
// by backward accumulation of the reflectors, and the implicit-shift QL
// iteration on the tridiagonal matrix (Bowdler, Martin, Reinsch & Wilkinson
// 1968) with the rotations accumulated into Q.  One CTA per block; the
// p x p working matrix lives in the block's eigenvector slot of the tape
// (global memory, column-major, L2-resident), so any p fits.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "kernels_psd.cuh"

namespace cosmo {

// shared scratch of the QL kernel: d, e, vh, wv, beta, rc, rs [p] T |
// sel [p + 2] int | red [2 nt/32] double
template <class T>
__host__ __device__ inline size_t tql_smem(int p, int nt) {
  return (size_t)7 * p * sizeof(T) + (size_t)(p + 8) * sizeof(int) + (size_t)(2 * (nt / 32)) * sizeof(double) + 64;
}
// the same with the p x p working matrix in shared memory too (after the
// scratch, 16-byte aligned): every phase then works on chip, and the
// eigenvectors are copied to the tape once at the end
template <class T>
__host__ __device__ inline size_t tql_smem_z(int p, int nt) {
  return ((tql_smem<T>(p, nt) + 15) & ~(size_t)15) + (size_t)p * p * sizeof(T);
}

// sum over the CTA of one double, broadcast (uses red[nt/32])
__device__ __forceinline__ double cta_sum1(double v, double* red) {
  double a[1] = {v};
  block_sum<1>(a, red);
  return a[0];
}

// Tridiagonalise the symmetric matrix Z (p x p, column-major, full storage)
// in place; on exit d (diagonal), e (e[k] couples k and k+1, e[p-1] = 0),
// reflector k (v, beta) stored in column k below the diagonal and beta[k].
template <class T>
__device__ void householder_tridiag(T* Z, int p, T* d, T* e, T* vh, T* wv, T* beta, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k + 2 < p; ++k) {
    const int n1 = p - k - 1;
    const T* col = Z + (size_t)k * p + k + 1;       // x = A[k+1:, k]
    double sq = 0.0;
    for (int i = tid; i < n1; i += nt) {
      const T x = col[i];
      vh[i] = x;
      if (i > 0) sq += (double)x * (double)x;
    }
    sq = cta_sum1(sq, red);
    const T x0 = vh[0];
    const T akk = Z[(size_t)k * p + k];
    T bet = T(0), alpha = x0;
    if (sq > 0.0) {
      const double nrm = sqrt((double)x0 * (double)x0 + sq);
      alpha = (T)(x0 >= T(0) ? -nrm : nrm);
      const T v0 = x0 - alpha;
      bet = (T)(2.0 / ((double)v0 * (double)v0 + sq));
      __syncthreads();
      if (tid == 0) vh[0] = v0;
    }
    __syncthreads();
    if (tid == 0) { d[k] = akk; e[k] = alpha; beta[k] = bet; }
    if (bet != T(0)) {
      // p = beta A_sub v (thread per row r of the trailing block; coalesced)
      double pv = 0.0;
      for (int r = tid; r < n1; r += nt) {
        // four partial sums (columns c = 0, 1, 2, 3 mod 4) break the FMA chain
        const T* zr = Z + (size_t)(k + 1) * p + (k + 1 + r);
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        int c = 0;
        for (; c + 3 < n1; c += 4) {
          a0 = fma(zr[(size_t)c * p], vh[c], a0);
          a1 = fma(zr[(size_t)(c + 1) * p], vh[c + 1], a1);
          a2 = fma(zr[(size_t)(c + 2) * p], vh[c + 2], a2);
          a3 = fma(zr[(size_t)(c + 3) * p], vh[c + 3], a3);
        }
        for (; c < n1; ++c) a0 = fma(zr[(size_t)c * p], vh[c], a0);
        const T acc = (a0 + a1) + (a2 + a3);
        const T pr = bet * acc;
        wv[r] = pr;
        pv += (double)pr * (double)vh[r];
      }
      pv = cta_sum1(pv, red);
      const T kc = (T)(0.5 * (double)bet * pv);
      for (int r = tid; r < n1; r += nt) wv[r] -= kc * vh[r];
      __syncthreads();
      // A_sub -= v w' + w v'
      for (int c = 0; c < n1; ++c) {
        const T vc = vh[c], wc = wv[c];
        T* colc = Z + (size_t)(k + 1 + c) * p + (k + 1);
        for (int r = tid; r < n1; r += nt) colc[r] -= vh[r] * wc + wv[r] * vc;
      }
    }
    // keep the reflector in column k (rows k+1..) for the formation of Q
    for (int i = tid; i < n1; i += nt) Z[(size_t)k * p + k + 1 + i] = (bet != T(0)) ? vh[i] : T(0);
    __syncthreads();
  }
  if (tid == 0) {
    if (p >= 2) {
      d[p - 2] = Z[(size_t)(p - 2) * p + (p - 2)];
      e[p - 2] = Z[(size_t)(p - 2) * p + (p - 1)];
      if (p == 2) beta[0] = T(0);
    }
    d[p - 1] = Z[(size_t)(p - 1) * p + (p - 1)];
    e[p - 1] = T(0);
  }
  __syncthreads();
}

// Q = H_0 H_1 ... H_{p-3} formed in place (reflector k in column k below the
// diagonal): Q^(k) = (I - beta_k v_k v_k') Q^(k+1), backwards from the
// identity; column and row k of Q^(k) are e_k.
template <class T>
__device__ void form_q(T* Z, int p, const T* beta, T* vh, T* wv) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  if (p >= 2) {
    if (tid == 0) {
      Z[(size_t)(p - 2) * p + (p - 2)] = T(1);
      Z[(size_t)(p - 1) * p + (p - 1)] = T(1);
      Z[(size_t)(p - 2) * p + (p - 1)] = T(0);
      Z[(size_t)(p - 1) * p + (p - 2)] = T(0);
    }
  } else if (tid == 0) {
    Z[0] = T(1);
  }
  __syncthreads();
  for (int k = p - 3; k >= 0; --k) {
    const int n1 = p - k - 1;
    const T bet = beta[k];
    for (int i = tid; i < n1; i += nt) vh[i] = Z[(size_t)k * p + k + 1 + i];
    __syncthreads();
    if (bet != T(0)) {
      // u_c = v' Q[k+1:, k+1+c]: four columns per warp at a time (their
      // warp reductions interleave), lanes over rows
      for (int c0 = 4 * w; c0 < n1; c0 += 4 * nw) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int r = lane; r < n1; r += 32) {
          const T vr = vh[r];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (c0 + q < n1) acc[q] = fma(vr, Z[(size_t)(k + 1 + c0 + q) * p + (k + 1) + r], acc[q]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        if (lane < 4 && c0 + lane < n1) {
          T a = acc[0];
#pragma unroll
          for (int q = 1; q < 4; ++q)
            if (lane == q) a = acc[q];
          wv[c0 + lane] = bet * a;
        }
      }
      __syncthreads();
      for (int c = 0; c < n1; ++c) {
        const T uc = wv[c];
        T* colc = Z + (size_t)(k + 1 + c) * p + (k + 1);
        for (int r = tid; r < n1; r += nt) colc[r] -= vh[r] * uc;
      }
    }
    // column k and row k become e_k
    for (int i = tid; i < p - k; i += nt) Z[(size_t)k * p + k + i] = (i == 0) ? T(1) : T(0);
    for (int c = k + 1 + tid; c < p; c += nt) Z[(size_t)c * p + k] = T(0);
    __syncthreads();
  }
}

template <class T> __device__ __forceinline__ T pythag_(T a, T b) { return hypot_(a, b); }

// The plane rotation of a QL step: r = hypot(f, g), s = f / r, c = g / r;
// false (r = 0) if f = g = 0.  (A reciprocal-square-root form with a Newton
// step was measured: the sweep got faster but the vertex-transitive Lovasz
// blocks, whose spectra are highly repeated, lost an order of magnitude of
// objective accuracy in FP32, so the IEEE quotients stay.)
template <class T>
__device__ __forceinline__ bool tql_rot(T f, T g, T& r, T& s, T& c) {
  r = pythag_(f, g);
  if (r == T(0)) return false;
  s = f / r;
  c = g / r;
  return true;
}

// Implicit-shift QL on the symmetric tridiagonal (d, e), rotations applied to
// the columns of Z (so Z Q_ql holds the eigenvectors).  Thread 0 runs the
// iteration and records each sweep's rotations (rc, rs for columns i, i+1,
// i from hi down to lo); all threads then apply them to their rows of Z with
// the running column in a register.  At most maxit sweeps per eigenvalue;
// returns false (and deflates) if that cap is hit.
template <class T>
__device__ bool tql_iterate(T* Z, int p, T* d, T* e, T* rc, T* rs, int* ctl, int maxit) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // thread 0 state
  int l = 0, iter = 0;
  bool ok = true;
  T tnorm = T(0);
  if (tid == 0) {
    for (int i = 0; i < p; ++i) tnorm = fmax(tnorm, fabs(d[i]) + fabs(e[i]));
  }
  const T eps = (T)Eps<T>::v;
  for (;;) {
    if (tid == 0) {
      int lo = 0, hi = -1, state = 0;
      while (l < p) {
        int m = l;
        for (; m < p - 1; ++m) {
          const T dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= eps * dd || fabs(e[m]) <= T(4) * eps * tnorm) break;
        }
        if (m == l) { ++l; iter = 0; continue; }
        if (++iter > maxit) { ok = false; e[l] = T(0); continue; }
        // shift from the leading 2 x 2 block
        T g = (d[l + 1] - d[l]) / (T(2) * e[l]);
        T r = pythag_(g, T(1));
        g = d[m] - d[l] + e[l] / (g + copysign(r, g));
        T s = T(1), c = T(1), pp = T(0);
        int i = m - 1;
        bool early = false;
        // step i reads e[i], d[i + 1], d[i] and writes e[i + 1], d[i + 1]:
        // d[i] and the next e, d are carried in registers (loaded ahead)
        T ei = e[i], di1 = d[i + 1], di = d[i];
        for (; i >= l; --i) {
          const T e_nx = i > l ? e[i - 1] : T(0), d_nx = i > l ? d[i - 1] : T(0);
          T f = s * ei;
          const T b = c * ei;
          if (!tql_rot(f, g, r, s, c)) {   // r = 0: deflation inside the sweep
            e[i + 1] = r;
            d[i + 1] = di1 - pp;
            e[m] = T(0);
            early = true;
            break;
          }
          e[i + 1] = r;
          g = di1 - pp;
          r = (di - g) * s + T(2) * c * b;
          pp = s * r;
          d[i + 1] = g + pp;
          g = c * r - b;
          rc[i] = c;
          rs[i] = s;
          ei = e_nx;
          di1 = di;
          di = d_nx;
        }
        if (!early) {
          d[l] -= pp;
          e[l] = g;
          e[m] = T(0);
          lo = l;
        } else {
          lo = i + 1;
        }
        hi = m - 1;
        state = 1;
        break;
      }
      ctl[0] = state;
      ctl[1] = lo;
      ctl[2] = hi;
    }
    __syncthreads();
    if (ctl[0] == 0) break;
    const int lo = ctl[1], hi = ctl[2];
    if (hi >= lo) {
      for (int k = tid; k < p; k += nt) {
        // rotation i acts on columns (i, i+1): z_{i+1} <- s z_i + c z_{i+1},
        // z_i <- c z_i - s z_{i+1}; i descends, so z_i carries to step i-1
        T f = Z[(size_t)(hi + 1) * p + k];
        for (int i = hi; i >= lo; --i) {
          const T zi = Z[(size_t)i * p + k];
          const T c = rc[i], s = rs[i];
          Z[(size_t)(i + 1) * p + k] = s * zi + c * f;
          f = c * zi - s * f;
        }
        Z[(size_t)lo * p + k] = f;
      }
    }
    __syncthreads();
  }
  if (tid == 0) ctl[3] = ok ? 1 : 0;
  __syncthreads();
  return ctl[3] != 0;
}

// a7 for large blocks: fused relaxation / projection / dual update like
// k_psd_fwd, with the tridiagonal + QL eigensolver.  zsm: the working matrix
// lives in shared memory (launched with tql_smem_z bytes) instead of the
// block's tape slot; the arithmetic and its order are the same either way.
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_psd_fwd_tql(Prob<T, V> P, PsdIterIO<T> io, T* lam_slot,
                                                    T* U_slot, int32_t* flags, int sched_off,
                                                    unsigned long long* stats, int maxit, int zsm) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = P.psd_sched[sched_off + blockIdx.x];
  const int p = P.psd_p[blk];
  const int64_t row0 = P.psd_row0[blk];
  T* d = reinterpret_cast<T*>(smraw);
  T* e = d + p;
  T* vh = e + p;
  T* wv = vh + p;
  T* beta = wv + p;
  T* rc = beta + p;
  T* rs = rc + p;
  int* ctl = reinterpret_cast<int*>(rs + p);
  int* sel = ctl + 8;
  double* red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(sel + p) + 7) & ~uintptr_t(7));
  const int inst = io.row_inst[row0];
  const T al = io.alpha[inst], rh = io.rho[row0];
  T* const Ut = U_slot + P.psd_uoff[blk];
  T* Z = zsm ? reinterpret_cast<T*>(smraw + ((tql_smem<T>(p, NT) + 15) & ~(size_t)15)) : Ut;
  // S (full, symmetric) into Z
  for (int q = threadIdx.x; q < p * p; q += NT) {
    const int j = q / p, i = q - j * p;
    const int a = min(i, j), b = max(i, j);
    const int64_t r = row0 + (int64_t)b * (b + 1) / 2 + a;
    T v = al * io.st[r] + (T(1) - al) * io.s[r] + io.y[r] / rh;
    if (a != b) v *= (T)kInvSqrt2;
    Z[(size_t)j * p + i] = v;
  }
  __syncthreads();
  householder_tridiag<T>(Z, p, d, e, vh, wv, beta, red);
  form_q<T>(Z, p, beta, vh, wv);
  const bool ok = tql_iterate<T>(Z, p, d, e, rc, rs, ctl, maxit);
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(&flags[inst], F_EIG_CAP);
    if (stats) { atomicAdd(&stats[1], 1ull); }
  }
  T* lam = lam_slot + P.psd_loff[blk];
  for (int k = threadIdx.x; k < p; k += NT) lam[k] = d[k];
  if (zsm)
    for (int q = threadIdx.x; q < p * p; q += NT) Ut[q] = Z[q];
  if (threadIdx.x == 0) {
    int npos = 0;
    for (int k = 0; k < p; ++k) npos += d[k] > T(0);
    const bool usepos = npos <= p - npos;
    int c = 0;
    for (int k = 0; k < p; ++k)
      if ((d[k] > T(0)) == usepos) sel[c++] = k;
    ctl[4] = c;
    ctl[5] = usepos;
  }
  __syncthreads();
  const int nsel = ctl[4];
  const bool usepos = ctl[5] != 0;
  const int dsv = p * (p + 1) / 2;
  for (int q = threadIdx.x; q < dsv; q += NT) {
    int i, j;
    svec_ij(q, i, j);
    T acc = T(0);
    for (int t = 0; t < nsel; ++t) {
      const int k = sel[t];
      acc += d[k] * Z[(size_t)k * p + i] * Z[(size_t)k * p + j];
    }
    const int64_t r = row0 + q;
    const T sh = al * io.st[r] + (T(1) - al) * io.s[r];
    T out;
    if (usepos) {
      out = acc;
    } else {
      T sij = sh + io.y[r] / rh;
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

// standalone batched projection with the tridiagonal + QL solver; the
// eigenvector output U (required) is the working matrix
template <class T, int NT>
__global__ void __launch_bounds__(NT) k_psd_project_tql(PsdBatch<T> B, const T* v, T* out,
                                                        T* lam_out, T* U_out, int maxit,
                                                        int32_t* flag) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int blk = blockIdx.x;
  const int p = B.p[blk];
  T* d = reinterpret_cast<T*>(smraw);
  T* e = d + p;
  T* vh = e + p;
  T* wv = vh + p;
  T* beta = wv + p;
  T* rc = beta + p;
  T* rs = rc + p;
  int* ctl = reinterpret_cast<int*>(rs + p);
  double* red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(ctl + 8 + p) + 7) & ~uintptr_t(7));
  const int64_t o = B.off[blk];
  T* Z = U_out + B.uoff[blk];
  for (int q = threadIdx.x; q < p * p; q += NT) {
    const int j = q / p, i = q - j * p;
    const int a = min(i, j), b = max(i, j);
    T x = v[o + (int64_t)b * (b + 1) / 2 + a];
    if (a != b) x *= (T)kInvSqrt2;
    Z[(size_t)j * p + i] = x;
  }
  __syncthreads();
  householder_tridiag<T>(Z, p, d, e, vh, wv, beta, red);
  form_q<T>(Z, p, beta, vh, wv);
  const bool ok = tql_iterate<T>(Z, p, d, e, rc, rs, ctl, maxit);
  if (!ok && threadIdx.x == 0 && flag) atomicOr(flag, F_EIG_CAP);
  if (lam_out)
    for (int k = threadIdx.x; k < p; k += NT) lam_out[B.loff[blk] + k] = d[k];
  const int dsv = p * (p + 1) / 2;
  for (int q = threadIdx.x; q < dsv; q += NT) {
    int i, j;
    svec_ij(q, i, j);
    T acc = T(0);
    for (int k = 0; k < p; ++k)
      if (d[k] > T(0)) acc += d[k] * Z[(size_t)k * p + i] * Z[(size_t)k * p + j];
    if (i != j) acc *= (T)kSqrt2;
    out[o + q] = acc;
  }
}

}  // namespace cosmo

namespace cosmo {

// C(i, j) = sum_k A(i, k) B(k, j) for p x p operands read through accessors
// (global memory), CTA-wide, 32 x 32 output tiles staged through shared
// memory sa, sb [32 x 33]; each thread owns 4 rows of one column of a tile.
template <class T, class LA, class LB, class F>
__device__ void cta_gemm_tiled(int p, LA a_at, LB b_at, F store, T* sa, T* sb) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int col = tid & 31, rg = tid >> 5;   // row group: rows rg*4 .. rg*4+3 (needs >= 8 warps)
  for (int ti = 0; ti < p; ti += 32) {
    for (int tj = 0; tj < p; tj += 32) {
      T acc[4] = {T(0), T(0), T(0), T(0)};
      for (int tk = 0; tk < p; tk += 32) {
        for (int q = tid; q < 32 * 32; q += nt) {
          const int r = q & 31, kk = q >> 5;
          const int gi = ti + r, gk = tk + kk;
          sa[r * 33 + kk] = (gi < p && gk < p) ? a_at(gi, gk) : T(0);
          const int gk2 = tk + r, gj = tj + kk;
          sb[r * 33 + kk] = (gk2 < p && gj < p) ? b_at(gk2, gj) : T(0);
        }
        __syncthreads();
        if (rg < 8) {
#pragma unroll 8
          for (int kk = 0; kk < 32; ++kk) {
            const T bv = sb[kk * 33 + col];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(sa[(rg * 4 + q) * 33 + kk], bv, acc[q]);
          }
        }
        __syncthreads();
      }
      if (rg < 8) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int gi = ti + rg * 4 + q, gj = tj + col;
          if (gi < p && gj < p) store(gi, gj, acc[q]);
        }
      }
    }
  }
}

// b3 (PSD) for blocks whose working set exceeds shared memory:
// out = svec(U (L o (U' smat(g) U)) U') with U, lambda from the tape and two
// p x p global scratch matrices W1, W2 per block (column-major).
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_psd_bwd_global(Prob<T, V> P, PsdBwdIO<T> io,
                                                       const T* lam_slot, const T* U_slot,
                                                       T* work, double dk_tau_rel, int sched_off) {
  __shared__ T sa[32 * 33], sb[32 * 33];
  __shared__ double smax;
  const int blk = P.psd_sched[sched_off + blockIdx.x];
  const int p = P.psd_p[blk];
  const int64_t row0 = P.psd_row0[blk];
  const T* lam = lam_slot + P.psd_loff[blk];
  const T* U = U_slot + P.psd_uoff[blk];
  T* W1 = work + 2 * P.psd_uoff[blk];
  T* W2 = W1 + (size_t)p * p;
  const T* g = io.g + row0;
  static_assert(NT >= 256, "tiled contraction assumes at least 8 warps");
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < p; ++k) m = fmax(m, fabs((double)lam[k]));
    smax = m;
  }
  __syncthreads();
  const double tau = dk_tau_rel * fmax(1.0, smax);
  auto tbar = [&](int i, int c) -> T {
    const int a = min(i, c), b = max(i, c);
    T v = g[(int64_t)b * (b + 1) / 2 + a];
    return a == b ? v : v * (T)kInvSqrt2;
  };
  // W1 = T_bar U
  cta_gemm_tiled<T>(p, tbar, [&](int c, int l) { return U[(size_t)l * p + c]; },
                    [&](int i, int l, T v) { W1[(size_t)l * p + i] = v; }, sa, sb);
  __syncthreads();
  // W2 = (U' W1) o L
  cta_gemm_tiled<T>(p, [&](int k, int i) { return U[(size_t)k * p + i]; },
                    [&](int i, int l) { return W1[(size_t)l * p + i]; },
                    [&](int k, int l, T v) {
                      W2[(size_t)l * p + k] = (T)((double)v * loewner_relu((double)lam[k], (double)lam[l], tau));
                    }, sa, sb);
  __syncthreads();
  // W1 = U W2
  cta_gemm_tiled<T>(p, [&](int i, int k) { return U[(size_t)k * p + i]; },
                    [&](int k, int l) { return W2[(size_t)l * p + k]; },
                    [&](int i, int l, T v) { W1[(size_t)l * p + i] = v; }, sa, sb);
  __syncthreads();
  const int dsv = p * (p + 1) / 2;
  for (int q = threadIdx.x; q < dsv; q += NT) {
    int i, j;
    svec_ij(q, i, j);
    T acc = T(0);
    for (int l = 0; l < p; ++l) acc = fma(W1[(size_t)l * p + i], U[(size_t)l * p + j], acc);
    if (i != j) acc *= (T)kSqrt2;
    io.vbar[row0 + q] = acc;
  }
}

}  // namespace cosmo
