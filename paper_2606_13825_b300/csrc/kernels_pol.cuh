// Closed-loop hyperparameter policy of App. E.  Step k of the unrolled
// iteration uses rho^k = exp(span sig(l^k_rho) + log rho_min) per row
// (span = log rho_max - log rho_min, [rho_min, rho_max] = [1e-3, 1e3]) and
// alpha^k = 2 sig(l^k_alpha) per instance; the logits follow
// l^{k+1} = l^k + MLP(xi^k) with two ReLU MLPs of 32x32 hidden units, one
// per constraint row on
//   xi_rho = [l_rho, s, y, rbar_p, log(||rbar_d||_inf + eps), delta_p, delta_d]
// and one per instance on
//   xi_alpha = [l_alpha, log(||rbar_p||_inf + eps), log(||rbar_d||_inf + eps),
//               log(||delta_p||_inf + eps), log(||delta_d||_inf + eps)],
// eps = 1e-12, the KKT residuals normalised OSQP-style (a zero scale counts
// as 1; r_d = P x + q - A'y), delta_d = s^k - s^{k-1}, delta_p = s^k - s~^k
// (both zero at k = 0).  The initial logits come per cone kind from l0 =
// (zero, orthant and box, soc, psd, alpha).
//
// The forward of step k's policy stores xi^k (feature-major over the
// flattened (k, row) index) and dMLP/dl (forward-mode through the ReLU
// masks), so that the reverse pass with the state features held constant is
// a per-row scan over k followed by the MLP reverse pass of kernels_ws.cuh.
#pragma once

#include "common.cuh"
#include "kernels_ws.cuh"

namespace cosmo {

constexpr int POL_H = 32;
constexpr int POL_NFR = 7;
constexpr int POL_NFA = 5;
constexpr double POL_LOG_RHO_MIN = -6.907755278982137;   // log(1e-3)
constexpr double POL_SPAN = 13.815510557964274;          // log(1e3) - log(1e-3)
constexpr double POL_EPS = 1e-12;

// the squash in the iterate type (FP64 throughput is a small fraction of
// FP32 on this part; the mixed-precision path keeps FP32 here)
template <class T>
__device__ inline T pol_sig(T z) { return T(1) / (T(1) + exp(-z)); }
template <class T>
__device__ inline T pol_rho(T l) { return exp(T(POL_SPAN) * pol_sig(l) + T(POL_LOG_RHO_MIN)); }
// slot of l0 for a cone kind: zero 0, orthant and box 1, soc 2, psd 3
__device__ inline int pol_slot(int kind) { return kind == 0 ? 0 : kind <= 2 ? 1 : kind == 3 ? 2 : 3; }

// MLP (F inputs, 32x32, one output) of one element, weights w in shared
// memory as ws_load_params lays them out (W2 transposed); J = d out / d x[0]
template <class T, int F>
__device__ __forceinline__ void pol_mlp(const T (&x)[F], const T* w, T& out, T& J) {
  const T *W1 = w, *b1 = W1 + F * POL_H, *W2 = b1 + POL_H, *b2 = W2 + POL_H * POL_H, *W3 = b2 + POL_H,
          *b3 = W3 + POL_H;
  T h[POL_H], t[POL_H];
#pragma unroll
  for (int i = 0; i < POL_H; ++i) {
    T z = b1[i];
#pragma unroll
    for (int f = 0; f < F; ++f) z += W1[f * POL_H + i] * x[f];
    h[i] = z > T(0) ? z : T(0);
    t[i] = z > T(0) ? W1[i] : T(0);
  }
  T o = b3[0], j1 = T(0);
#pragma unroll 1
  for (int j = 0; j < POL_H; ++j) {
    // W2 transposed in shared memory (ws_load_params): row j is column j
    const T z = ws_dot<T, POL_H>(b2[j], W2 + j * POL_H, h);
    const T dz = ws_dot<T, POL_H>(T(0), W2 + j * POL_H, t);
    if (z > T(0)) {
      o += W3[j] * z;
      j1 += W3[j] * dz;
    }
  }
  out = o;
  J = j1;
}

// l^0, rho^0 per row and l^0_alpha, alpha^0 per instance from l0 [5]
template <class T, class V>
__global__ void k_pol_init(Prob<T, V> P, const T* __restrict__ l0, T* __restrict__ lr, T* __restrict__ rho,
                           T* __restrict__ la, T* __restrict__ alpha) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < P.m_total) {
    const T l = l0[pol_slot(P.row_kind[e])];
    lr[e] = l;
    rho[e] = pol_rho(l);
  }
  if (e < P.ninst) {
    la[e] = l0[4];
    alpha[e] = T(2) * pol_sig(l0[4]);
  }
}

// per instance (one CTA): the infinity norms of the features, the instance
// scalars 1/scale_p and log(||rbar_d|| + eps) for the row kernel, and the
// alpha MLP: l^{k+1}_alpha, alpha^{k+1}, xi_alpha^k, dMLP/dl
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_pol_inst(Prob<T, V> P, const T* __restrict__ x, const T* __restrict__ s,
                                                 const T* __restrict__ y, const T* __restrict__ sprev,
                                                 const T* __restrict__ stil, const T* __restrict__ theta,
                                                 const T* __restrict__ la, T* __restrict__ la_next,
                                                 T* __restrict__ alpha_next, T* __restrict__ Xa, int64_t lda,
                                                 T* __restrict__ Ja, T* __restrict__ sc) {
  __shared__ double sm[10][NT / 32];
  const int32_t inst = blockIdx.x;
  const int64_t c0 = P.col_off[inst], c1 = P.col_off[inst + 1];
  const int64_t r0 = P.row_off[inst], r1 = P.row_off[inst + 1];
  // r_p, Ax, s, b, r_d, Px, q, A'y, delta_p, delta_d: maxima of |.| in the
  // iterate type (exact: a maximum does not round), widened at the end
  T v[10] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  for (int64_t r = r0 + threadIdx.x; r < r1; r += NT) {
    T ax = T(0);
    for (int64_t e = P.A_rp[r]; e < P.A_rp[r + 1]; ++e) ax += (T)ldv(P.A_v, e) * x[P.A_ci[e]];
    v[0] = fmax(v[0], fabs(ax + s[r] - P.b[r]));
    v[1] = fmax(v[1], fabs(ax));
    v[2] = fmax(v[2], fabs(s[r]));
    v[3] = fmax(v[3], fabs(P.b[r]));
    if (stil) v[8] = fmax(v[8], fabs(s[r] - stil[r]));
    if (sprev) v[9] = fmax(v[9], fabs(s[r] - sprev[r]));
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
  for (int k = 0; k < 10; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = fmax(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    if (lane == 0) sm[k][w] = (double)v[k];
  }
  __syncthreads();
  if (w != 0) return;
  // warp 0: every lane forms the same norms and features; lane j then owns
  // hidden unit j of both layers of the alpha MLP (32 units)
  double vd[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    double mx = 0.0;
    for (int q = 0; q < NT / 32; ++q) mx = fmax(mx, sm[k][q]);
    vd[k] = mx;
  }
  double scp = fmax(fmax(vd[1], vd[2]), vd[3]), scd = fmax(fmax(vd[5], vd[6]), vd[7]);
  scp = scp > 0.0 ? scp : 1.0;
  scd = scd > 0.0 ? scd : 1.0;
  const double lgd = log(vd[4] / scd + POL_EPS);
  const T xi[POL_NFA] = {la[inst], (T)log(vd[0] / scp + POL_EPS), (T)lgd, (T)log(vd[8] + POL_EPS),
                         (T)log(vd[9] + POL_EPS)};
  if (lane == 0) {
    sc[inst] = (T)(1.0 / scp);
    sc[P.ninst + inst] = (T)lgd;
  }
  if (lane < POL_NFA) Xa[lane * lda + inst] = xi[lane];
  const T *W1 = theta, *b1 = W1 + POL_NFA * POL_H, *W2 = b1 + POL_H, *b2 = W2 + POL_H * POL_H, *W3 = b2 + POL_H,
          *b3 = W3 + POL_H;
  T z1 = b1[lane];
#pragma unroll
  for (int f = 0; f < POL_NFA; ++f) z1 += W1[f * POL_H + lane] * xi[f];
  const T h1 = z1 > T(0) ? z1 : T(0), t1 = z1 > T(0) ? W1[lane] : T(0);
  T z2 = b2[lane], dz2 = T(0);
#pragma unroll 8
  for (int i = 0; i < POL_H; ++i) {
    const T hi = __shfl_sync(0xffffffffu, h1, i), ti = __shfl_sync(0xffffffffu, t1, i);
    z2 += W2[i * POL_H + lane] * hi;
    dz2 += W2[i * POL_H + lane] * ti;
  }
  T o = z2 > T(0) ? W3[lane] * z2 : T(0), J = z2 > T(0) ? W3[lane] * dz2 : T(0);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    o += __shfl_xor_sync(0xffffffffu, o, d);
    J += __shfl_xor_sync(0xffffffffu, J, d);
  }
  if (lane == 0) {
    const T l = la[inst] + b3[0] + o;
    la_next[inst] = l;
    alpha_next[inst] = T(2) * pol_sig(l);
    Ja[inst] = J;
  }
}

// per row (thread per row, 128 per CTA): xi_rho^k, the rho MLP, l^{k+1},
// rho^{k+1} (before rectification), dMLP/dl
template <class T, class V>
__global__ void __launch_bounds__(128) k_pol_rows(Prob<T, V> P, const T* __restrict__ x, const T* __restrict__ s,
                                                  const T* __restrict__ y, const T* __restrict__ sprev,
                                                  const T* __restrict__ stil, const T* __restrict__ theta,
                                                  const T* __restrict__ lr, T* __restrict__ lr_next,
                                                  T* __restrict__ rho_next, T* __restrict__ Xr, int64_t ldr,
                                                  T* __restrict__ Jr, const T* __restrict__ sc) {
  extern __shared__ __align__(16) unsigned char pol_sm[];
  const T* w = ws_load_params<T, POL_NFR, 1, POL_H>(theta, reinterpret_cast<T*>(pol_sm));
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= P.m_total) return;
  const int i = P.row_inst[r];
  T ax = T(0);
  for (int64_t e = P.A_rp[r]; e < P.A_rp[r + 1]; ++e) ax += (T)ldv(P.A_v, e) * x[P.A_ci[e]];
  const T sr = s[r];
  T xi[POL_NFR] = {lr[r], sr, y[r], (ax + sr - P.b[r]) * sc[i], sc[P.ninst + i], stil ? sr - stil[r] : T(0),
                   sprev ? sr - sprev[r] : T(0)};
#pragma unroll
  for (int f = 0; f < POL_NFR; ++f) Xr[f * ldr + r] = xi[f];
  T out, J;
  pol_mlp<T, POL_NFR>(xi, w, out, J);
  const T l = lr[r] + out;
  lr_next[r] = l;
  rho_next[r] = pol_rho(l);
  Jr[r] = J;
}

// reverse scan over the steps, thread per element e < N (rows, or
// instances when ALPHA): with g the cotangent of l^{k+1},
//   G[k][e] = g (the cotangent of the MLP output at step k, k < K - 1),
//   g <- g (1 + J[k][e]) + gp[k][e] dp/dl (l^k[e])
// where p = rho (squashed) or alpha; gl0[e] = g at the end
// (p = the stored rho or alpha of each step: drho/dl = rho span sig (1 -
// sig), dalpha/dl = 2 sig (1 - sig); g carried in double)
template <class T, bool ALPHA>
__global__ void k_pol_scan(int32_t K, int64_t N, const T* __restrict__ gp, const T* __restrict__ p,
                           const T* __restrict__ l, const T* __restrict__ J, T* __restrict__ G, T* __restrict__ gl0) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N) return;
  double g = 0.0;
  for (int32_t k = K - 1; k >= 0; --k) {
    const int64_t o = (int64_t)k * N + e;
    if (k + 1 < K) {
      G[o] = (T)g;
      g *= 1.0 + (double)J[o];
    }
    const T sg = pol_sig(l[o]);
    const T dp = (ALPHA ? T(2) : p[o] * T(POL_SPAN)) * sg * (T(1) - sg);
    g += (double)gp[o] * (double)dp;
  }
  gl0[e] = (T)g;
}

// gl0[0..3] = sums of the rows' l^0 cotangents by slot, gl0[4] = sum over
// instances (one CTA of 256 threads, fixed order)
template <class T, class V>
__global__ void __launch_bounds__(256) k_pol_l0(Prob<T, V> P, const T* __restrict__ glr, const T* __restrict__ gla,
                                                T* __restrict__ gl0) {
  __shared__ double sm[5][256];
  double a[5] = {0, 0, 0, 0, 0};
  for (int64_t r = threadIdx.x; r < P.m_total; r += 256) a[pol_slot(P.row_kind[r])] += (double)glr[r];
  for (int64_t i = threadIdx.x; i < P.ninst; i += 256) a[4] += (double)gla[i];
#pragma unroll
  for (int q = 0; q < 5; ++q) sm[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h)
#pragma unroll
      for (int q = 0; q < 5; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 5) gl0[threadIdx.x] = (T)sm[threadIdx.x][0];
}

}  // namespace cosmo
