// Warm-start network of App. E: the initial iterate predicted elementwise by
// two shared ReLU MLPs (two hidden layers of width 64), one per decision
// variable from phi_j = [q_j, P_jj, ||A_{:,j}||_2, nnz(A_{:,j}), ctx], one per
// constraint row from psi_r = [b_r, ||A_{r,:}||_2, nnz(A_{r,:}), onehot(cone of
// r), ctx], with the instance context ctx = (log(1 + ||q||_inf), log(1 +
// ||b||_inf), log(1 + n_i), log(1 + m_i)).
//
// Parameters of an MLP with F inputs and O outputs, flattened: W1 [F][64],
// b1 [64], W2 [64][64], b2 [64], W3 [64][O], b3 [O]; a layer is
// h = relu(W' u + b).  Features are stored feature-major ([F][N]) so that a
// thread per element reads them coalesced.  The forward and the per-element
// reverse pass keep a hidden layer (64 values) in registers and the weights
// in shared memory (every lane reads the same weight: a broadcast).  The
// weight gradients are sums over elements of outer products; they are formed
// by a chunked reduction in a fixed order (bitwise reproducible).
#pragma once

#include "common.cuh"

namespace cosmo {

constexpr int WS_H = 64;
constexpr int WS_NFX = 8;
constexpr int WS_NFC = 12;
__host__ __device__ constexpr int ws_nparams(int F, int O, int H = WS_H) { return F * H + H + H * H + H + H * O + O; }

// ctx[4 i + k] of instance i (one CTA per instance; maxima in double)
template <class T, class V, int NT>
__global__ void __launch_bounds__(NT) k_ws_ctx(Prob<T, V> P, T* __restrict__ ctx) {
  __shared__ double sm[2][NT / 32];
  const int i = blockIdx.x;
  const int64_t c0 = P.col_off[i], c1 = P.col_off[i + 1], r0 = P.row_off[i], r1 = P.row_off[i + 1];
  double qm = 0.0, bm = 0.0;
  for (int64_t j = c0 + threadIdx.x; j < c1; j += NT) qm = fmax(qm, fabs((double)P.q[j]));
  for (int64_t r = r0 + threadIdx.x; r < r1; r += NT) bm = fmax(bm, fabs((double)P.b[r]));
  for (int o = 16; o > 0; o >>= 1) {
    qm = fmax(qm, __shfl_xor_sync(0xffffffffu, qm, o));
    bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
  }
  if ((threadIdx.x & 31) == 0) { sm[0][threadIdx.x >> 5] = qm; sm[1][threadIdx.x >> 5] = bm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; ++w) { qm = fmax(qm, sm[0][w]); bm = fmax(bm, sm[1][w]); }
    ctx[4 * i + 0] = (T)log1p(qm);
    ctx[4 * i + 1] = (T)log1p(bm);
    ctx[4 * i + 2] = (T)log1p((double)(c1 - c0));
    ctx[4 * i + 3] = (T)log1p((double)(r1 - r0));
  }
}

// FX [8][n] and FC [12][m] (feature-major)
template <class T, class V>
__global__ void k_ws_feat(Prob<T, V> P, const T* __restrict__ ctx, T* __restrict__ FX, T* __restrict__ FC) {
  const int64_t n = P.n_total, m = P.m_total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n + m; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < n) {
      const int64_t j = e;
      const int i = P.col_inst[j];
      double cn = 0.0;
      for (int64_t k = P.AT_rp[j]; k < P.AT_rp[j + 1]; ++k) {
        const double a = (double)ldv(P.AT_v, k);
        cn += a * a;
      }
      FX[0 * n + j] = P.q[j];
      FX[1 * n + j] = P.Pdiag[j];
      FX[2 * n + j] = (T)sqrt(cn);
      FX[3 * n + j] = (T)(P.AT_rp[j + 1] - P.AT_rp[j]);
      for (int k = 0; k < 4; ++k) FX[(4 + k) * n + j] = ctx[4 * i + k];
    } else {
      const int64_t r = e - n;
      const int i = P.row_inst[r];
      double rn = 0.0;
      for (int64_t k = P.A_rp[r]; k < P.A_rp[r + 1]; ++k) {
        const double a = (double)ldv(P.A_v, k);
        rn += a * a;
      }
      FC[0 * m + r] = P.b[r];
      FC[1 * m + r] = (T)sqrt(rn);
      FC[2 * m + r] = (T)(P.A_rp[r + 1] - P.A_rp[r]);
      const int kind = P.row_kind[r];
      for (int k = 0; k < 5; ++k) FC[(3 + k) * m + r] = kind == k ? T(1) : T(0);
      for (int k = 0; k < 4; ++k) FC[(8 + k) * m + r] = ctx[4 * i + k];
    }
  }
}

// the parameters into shared memory (all threads of the CTA), with W2
// stored transposed (row j of the copy = column j of W2: the inner loops
// over i read it with 16-byte vector loads)
template <class T, int F, int O, int H = WS_H>
__device__ __forceinline__ T* ws_load_params(const T* __restrict__ theta, T* sm) {
  constexpr int o2 = F * H + H;
  for (int k = threadIdx.x; k < ws_nparams(F, O, H); k += blockDim.x) {
    const int d = k - o2;
    sm[(d >= 0 && d < H * H) ? o2 + (d % H) * H + d / H : k] = theta[k];
  }
  __syncthreads();
  return sm;
}

// z + sum_i w[i] h[i] in order of i (w: 16-byte aligned shared memory)
template <class T, int H>
__device__ __forceinline__ T ws_dot(T z, const T* w, const T (&h)[H]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int q = 0; q < H / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(w)[q];
      z += v.x * h[4 * q];
      z += v.y * h[4 * q + 1];
      z += v.z * h[4 * q + 2];
      z += v.w * h[4 * q + 3];
    }
  } else {
#pragma unroll
    for (int q = 0; q < H / 2; ++q) {
      const double2 v = reinterpret_cast<const double2*>(w)[q];
      z += v.x * h[2 * q];
      z += v.y * h[2 * q + 1];
    }
  }
  return z;
}

// h[i] += w[i] d for every i (w: 16-byte aligned shared memory)
template <class T, int H>
__device__ __forceinline__ void ws_axpy(T (&h)[H], const T* w, T d) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int q = 0; q < H / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(w)[q];
      h[4 * q] += v.x * d;
      h[4 * q + 1] += v.y * d;
      h[4 * q + 2] += v.z * d;
      h[4 * q + 3] += v.w * d;
    }
  } else {
#pragma unroll
    for (int q = 0; q < H / 2; ++q) {
      const double2 v = reinterpret_cast<const double2*>(w)[q];
      h[2 * q] += v.x * d;
      h[2 * q + 1] += v.y * d;
    }
  }
}

// h1 = relu(W1' x + b1) of element e (features X[f * ld + e])
template <class T, int F, int H = WS_H>
__device__ __forceinline__ void ws_layer1(const T* __restrict__ X, int64_t ld, int64_t e, const T* W1, const T* b1,
                                          T (&h1)[H]) {
  T x[F];
#pragma unroll
  for (int f = 0; f < F; ++f) x[f] = X[f * ld + e];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    T z = b1[i];
#pragma unroll
    for (int f = 0; f < F; ++f) z += W1[f * H + i] * x[f];
    h1[i] = z > T(0) ? z : T(0);
  }
}

// out[o][e] for every element (thread per element; up to two outputs)
template <class T, int F, int O>
__global__ void __launch_bounds__(128) k_ws_fwd(int64_t N, const T* __restrict__ X, const T* __restrict__ theta,
                                                T* __restrict__ out0, T* __restrict__ out1) {
  extern __shared__ __align__(16) unsigned char ws_sm[];
  const T* w = ws_load_params<T, F, O>(theta, reinterpret_cast<T*>(ws_sm));
  const T *W1 = w, *b1 = W1 + F * WS_H, *W2 = b1 + WS_H, *b2 = W2 + WS_H * WS_H, *W3 = b2 + WS_H, *b3 = W3 + WS_H * O;
  // one element per thread: in a grid-stride loop the compiler hoists the
  // loop-invariant weight reads into registers and spills
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < N) {
    T h1[WS_H];
    ws_layer1<T, F>(X, N, e, W1, b1, h1);
    T o0 = b3[0], o1 = O > 1 ? b3[O - 1] : T(0);
#pragma unroll 1
    for (int j = 0; j < WS_H; ++j) {
      const T z = ws_dot<T, WS_H>(b2[j], W2 + j * WS_H, h1);   // W2 transposed in shared memory
      if (z > T(0)) {
        o0 += W3[j * O] * z;
        if (O > 1) o1 += W3[j * O + 1] * z;
      }
    }
    out0[e] = o0;
    if (O > 1) out1[e] = o1;
  }
}

// reverse pass per element e < N, for the cotangent G[o * ldg + e] of the
// outputs, features X[f * ldx + e]: H1 = relu(z1), D1 = dL/dz1, H2 =
// relu(z2), D2 = dL/dz2, each [H][N]
template <class T, int F, int O, int H = WS_H>
__global__ void __launch_bounds__(128) k_ws_bwd(int64_t N, int64_t ldx, const T* __restrict__ X,
                                                const T* __restrict__ theta, const T* __restrict__ G, int64_t ldg,
                                                T* __restrict__ H1, T* __restrict__ D1, T* __restrict__ H2,
                                                T* __restrict__ D2) {
  extern __shared__ __align__(16) unsigned char ws_sm[];
  const T* w = ws_load_params<T, F, O, H>(theta, reinterpret_cast<T*>(ws_sm));
  const T *W1 = w, *b1 = W1 + F * H, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H;
  // Two phases so that at most 64 values of a thread are live (fp64 would
  // spill with h1 and d2 both in registers): the layer-2 cotangent goes to
  // D2 and is read back by the same thread for layer 1.
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < N) {
    T h[H];
    ws_layer1<T, F, H>(X, ldx, e, W1, b1, h);
    T g[O];
#pragma unroll
    for (int o = 0; o < O; ++o) g[o] = G[o * ldg + e];
#pragma unroll 1
    for (int j = 0; j < H; ++j) {
      const T z = ws_dot<T, H>(b2[j], W2 + j * H, h);   // W2 transposed in shared memory
      T gz = T(0);
#pragma unroll
      for (int o = 0; o < O; ++o) gz += W3[j * O + o] * g[o];
      H2[j * N + e] = z > T(0) ? z : T(0);
      D2[j * N + e] = z > T(0) ? gz : T(0);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) H1[i * N + e] = h[i];
    // h now accumulates W2 d2
#pragma unroll
    for (int i = 0; i < H; ++i) h[i] = T(0);
#pragma unroll 1
    for (int j = 0; j < H; ++j) {
      ws_axpy<T, H>(h, W2 + j * H, D2[j * N + e]);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) D1[i * N + e] = H1[i * N + e] > T(0) ? h[i] : T(0);   // [z1 > 0] = [h1 > 0]
  }
}

constexpr int WS_MAXCH = 148 * 4;   // CTAs of the weight-gradient reduction: 4 per SM
constexpr int WS_TILE = 32;      // elements staged in shared memory at a time

// part[c][a * KB + b] = sum over elements n of chunk c (elements c * chunk
// up to (c + 1) * chunk, chunk a multiple of 32) of A'[a][n] B[b][n]
// (rows lda, ldb apart), where A' is A [KA][N] with a row of ones appended
// when `ones` is set (the bias gradient lands right after the weight
// gradient, as in the parameter layout), B [KB][N]; KA + ones <= RI * TY,
// KB <= RJ * TX (at most 80 x 64).  256 threads as G = 256 / (TY TX) groups
// of TY x TX: thread (g, ty, tx) owns rows ty + TY i (i < RI) and columns
// tx + TX j (j < RJ) and takes the elements t = g, g + G, ... of each staged
// 32-element tile, summed in T per tile and then in double; the G group
// partials are added in group order at the end (bitwise reproducible).  The
// shape (RI, RJ, TY, TX) is picked per output size so that few threads idle.
template <class T, int RI, int RJ, int TY, int TX>
__global__ void __launch_bounds__(256) k_ws_atb(int64_t N, int64_t chunk, const T* __restrict__ A, int64_t lda,
                                                int KA, int ones, const T* __restrict__ B, int64_t ldb, int KB,
                                                double* __restrict__ part) {
  constexpr int G = 256 / (TY * TX), NR = RI * TY, NC = RJ * TX;
  static_assert(G * TY * TX == 256 && NR <= 80 && NC <= 64, "thread shape");
  constexpr int RA = 81, RB = 65;   // odd row lengths: the transposing stores are conflict-free
  __shared__ __align__(16) unsigned char atb_sm[sizeof(T) * WS_TILE * (RA + RB)];
  T(*sa)[RA] = reinterpret_cast<T(*)[RA]>(atb_sm);
  T(*sb)[RB] = reinterpret_cast<T(*)[RB]>(atb_sm + sizeof(T) * WS_TILE * RA);
  const int64_t n0 = (int64_t)blockIdx.x * chunk, n1 = min(N, n0 + chunk);
  const int ka = KA + ones;
  const int g = threadIdx.x / (TY * TX), l = threadIdx.x % (TY * TX), ty = l / TX, tx = l % TX;
  double acc[RI][RJ];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < RJ; ++j) acc[i][j] = 0.0;
  for (int64_t t0 = n0; t0 < n1; t0 += WS_TILE) {
    const int tl = (int)min((int64_t)WS_TILE, n1 - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < NR * WS_TILE; k += 256) {
      const int a = k / WS_TILE, t = k % WS_TILE;
      sa[t][a] = (a < ka && t < tl) ? (a < KA ? A[a * lda + t0 + t] : T(1)) : T(0);
    }
    for (int k = threadIdx.x; k < NC * WS_TILE; k += 256) {
      const int b = k / WS_TILE, t = k % WS_TILE;
      sb[t][b] = (b < KB && t < tl) ? B[b * ldb + t0 + t] : T(0);
    }
    __syncthreads();
    T s[RI][RJ];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < RJ; ++j) s[i][j] = T(0);
#pragma unroll 4
    for (int t = g; t < WS_TILE; t += G) {
      T av[RI], bv[RJ];
#pragma unroll
      for (int i = 0; i < RI; ++i) av[i] = sa[t][ty + TY * i];
#pragma unroll
      for (int j = 0; j < RJ; ++j) bv[j] = sb[t][tx + TX * j];
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < RJ; ++j) s[i][j] += av[i] * bv[j];
    }
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < RJ; ++j) acc[i][j] += (double)s[i][j];
  }
  const int npair = ka * KB;
  if (G > 1) {
    // group partials through shared memory (the staging buffers), summed in group order
    static_assert(G == 1 || (size_t)G * NR * NC * sizeof(double) <= sizeof(atb_sm), "reduction space");
    double* red = reinterpret_cast<double*>(atb_sm);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < RJ; ++j) red[(g * NR + ty + TY * i) * NC + tx + TX * j] = acc[i][j];
    __syncthreads();
    for (int k = threadIdx.x; k < NR * NC; k += 256) {
      const int a = k / NC, b = k % NC;
      if (a < ka && b < KB) {
        double v = 0.0;
        for (int q = 0; q < G; ++q) v += red[(q * NR + a) * NC + b];
        part[(int64_t)blockIdx.x * npair + a * KB + b] = v;
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < RJ; ++j) {
      const int a = ty + TY * i, b = tx + TX * j;
      if (a < ka && b < KB) part[(int64_t)blockIdx.x * npair + a * KB + b] = acc[i][j];
    }
}

// The weight sums of a thin block (KB <= 2 columns: the output layers),
// part[c][a * KB + b] = sum over the elements n of chunk c of A'[a][n] B[b][n]
// with A' = [A; 1]: every thread streams its elements (n = n0 + tid, + 256,
// ...) with coalesced reads, 16 rows of A' at a time held in registers,
// sums in T per thread and over the warp (butterfly), then in double over
// the eight warps in warp order (bitwise reproducible).
template <class T>
__global__ void __launch_bounds__(256) k_ws_atb_thin(int64_t N, int64_t chunk, const T* __restrict__ A, int64_t lda,
                                                     int KA, int ones, const T* __restrict__ B, int64_t ldb, int KB,
                                                     double* __restrict__ part) {
  constexpr int RB = 16;
  __shared__ double sm[8][RB * 2];
  const int64_t n0 = (int64_t)blockIdx.x * chunk, n1 = min(N, n0 + chunk);
  const int ka = KA + ones, npair = ka * KB, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* out = part + (int64_t)blockIdx.x * npair;
  for (int a0 = 0; a0 < ka; a0 += RB) {
    T acc[RB][2];
#pragma unroll
    for (int i = 0; i < RB; ++i) acc[i][0] = acc[i][1] = T(0);
    for (int64_t n = n0 + threadIdx.x; n < n1; n += 256) {
      const T g0 = B[n], g1 = KB > 1 ? B[ldb + n] : T(0);
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const int a = a0 + i;
        const T x = a < KA ? A[a * lda + n] : (a < ka ? T(1) : T(0));
        acc[i][0] += x * g0;
        acc[i][1] += x * g1;
      }
    }
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int b = 0; b < 2; ++b)
        if (b < KB) {   // warp butterfly in T (full-rate pipe), the warps combined in double
          const T v = warp_allsum(acc[i][b]);
          if (lane == 0) sm[w][2 * i + b] = (double)v;
        }
    __syncthreads();
    if (threadIdx.x < 2 * RB) {
      const int i = threadIdx.x >> 1, b = threadIdx.x & 1, a = a0 + i;
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) v += sm[q][threadIdx.x];
      if (a < ka && b < KB) out[a * KB + b] = v;
    }
    __syncthreads();
  }
}

// out[k] (+)= sum over chunks c of part[c][k]: 32 outputs per CTA of 256
// threads, warp q adding the chunks c = q, q + 8, ... in order, then the
// eight warp sums added in warp order (a fixed order: bitwise reproducible)
template <class T>
__global__ void __launch_bounds__(256) k_ws_sum(int nchunk, int npair, const double* __restrict__ part,
                                                T* __restrict__ out, int accumulate) {
  __shared__ double sm[8][32];
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5, k = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (k < npair)
    for (int c = q; c < nchunk; c += 8) s += part[(int64_t)c * npair + k];
  sm[q][lane] = s;
  __syncthreads();
  if (q == 0 && k < npair) {
    double v = accumulate ? (double)out[k] : 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += sm[w][lane];
    out[k] = (T)v;
  }
}

}  // namespace cosmo
