// Slot-layout cyclic Jacobi with a compile-time shared-memory geometry (the
// eigensolver of the PSD projection, Sec. 2.4, Eq. psd-proj), and the
// projection kernel built on it.
//
// The ordering, the 2x2 tiles in four planes, the fixed slot permutation and
// the pair role are those of kernels_jt.cuh (Brent & Luk round-robin; Golub &
// Van Loan Alg. 8.5.1 for the 2x2 rotation).  What changes is how a round is
// issued.  The block's geometry is fixed per size class (orders up to PMAX):
// plane, buffer and row strides are compile-time constants, so every shared
// access of a round is one register plus an immediate offset.  The tiles and
// the eigenvectors are double-buffered and the round is instantiated once
// per buffer parity, so the current / next buffers are immediates too.  The
// eigenvectors are kept by *slot*: row s of the V buffer is the vector of
// the index that slot s holds, and a round rotates the two rows of each pair
// and writes them to the rows the slot permutation gives them in the next
// round (after a whole number of sweeps every index is back in its first
// slot, so the vectors return to index order with one copy).  A thread's
// work items are fixed for the whole solve: up to TI off-diagonal tiles
// (seven byte offsets each: source, two rotations, four destinations) and up
// to CI eigenvector chunks (two 16-byte vectors of the pair's two rows:
// source, two destinations, rotation), in separate loops.
#pragma once

#include "kernels_psd.cuh"

namespace cosmo {

template <class T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

__device__ __forceinline__ void jt2_rotv(float4& a, float4& b, JtRot<float> r) {
  const float4 x = a, y = b;
  a = make_float4(jt_cms(r.c, r.s, x.x, y.x), jt_cms(r.c, r.s, x.y, y.y), jt_cms(r.c, r.s, x.z, y.z),
                  jt_cms(r.c, r.s, x.w, y.w));
  b = make_float4(jt_spc(r.c, r.s, x.x, y.x), jt_spc(r.c, r.s, x.y, y.y), jt_spc(r.c, r.s, x.z, y.z),
                  jt_spc(r.c, r.s, x.w, y.w));
}
__device__ __forceinline__ void jt2_rotv(double2& a, double2& b, JtRot<double> r) {
  const double2 x = a, y = b;
  a = make_double2(jt_cms(r.c, r.s, x.x, y.x), jt_cms(r.c, r.s, x.y, y.y));
  b = make_double2(jt_spc(r.c, r.s, x.x, y.x), jt_spc(r.c, r.s, x.y, y.y));
}

// C = A B for A with 16-byte-aligned rows contiguous along k (the eigenvector
// rows Vt): the warp-strided mapping of smem_gemm_w (warp w owns rows
// w + TY a, lane owns columns lane + 32 b), A read a 16-byte vector (four
// or two k) at a time.  The sum runs over k in the same order with the same
// fused multiply-adds, so the result is the one smem_gemm_w gives.
template <class T, int TM, int TN, class F>
__device__ __forceinline__ void jt2_gemm_w(int p, const T* A, int ar, const T* B, int br, int bc, F f) {
  using VT = typename Vec16<T>::type;
  constexpr int VL = 16 / (int)sizeof(T);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, TY = blockDim.x >> 5;
  const int pk = p & ~(VL - 1);
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
      int k = 0;
      for (; k < pk; k += VL) {
        T av[TM][VL];
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          const VT v = *reinterpret_cast<const VT*>(A + ii[a] * ar + k);
          const T* c = reinterpret_cast<const T*>(&v);
#pragma unroll
          for (int q = 0; q < VL; ++q) av[a][q] = c[q];
        }
#pragma unroll
        for (int q = 0; q < VL; ++q) {
          T bv[TN];
#pragma unroll
          for (int b = 0; b < TN; ++b) bv[b] = B[(k + q) * br + jj[b] * bc];
#pragma unroll
          for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) acc[a][b] = fma(av[a][q], bv[b], acc[a][b]);
        }
      }
      for (; k < p; ++k) {
        T av[TM], bv[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = A[ii[a] * ar + k];
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
template <class T, class F>
__device__ __forceinline__ void jt2_gemm(int p, const T* A, int ar, const T* B, int br, int bc, F f) {
  if constexpr (sizeof(T) == 8) {   // FP64: the scalar form (the vector one spills at 64 registers)
    smem_gemm_auto<T>(p, A, ar, 1, B, br, bc, f);
    return;
  }
  if (blockDim.x >= 512) jt2_gemm_w<T, 5, 3>(p, A, ar, B, br, bc, f);
  else if (blockDim.x >= 256) jt2_gemm_w<T, 7, 2>(p, A, ar, B, br, bc, f);
  else jt2_gemm_w<T, 8, 1>(p, A, ar, B, br, bc, f);
}

// Geometry for orders p <= PMAX (byte offsets from the dynamic shared base):
//   V   [2][PE][LDV]  eigenvectors by row, two buffers (index order outside
//                     the solve, slot order inside it)
//   S   [PE][LDS]     the block and the products' outputs
//   T   [2][4][PS]    tile buffers (four planes each); outside the solve the
//                     product buffer X (PE x LDS fits: asserted)
//   R   [2][NPM]      rotations of the current and the next round
//   L   [PE]          eigenvalues, the selected index set [PE + 2] int, then
//                     the reduction scratch (doubles)
template <class T, int PMAX>
struct Jt2Geo {
  static constexpr int PE = PMAX + (PMAX & 1);
  static constexpr int NPM = PE / 2;
  static constexpr int PS = ((NPM * (NPM + 1) / 2) + 31) & ~31;
  static constexpr int TBUF = 4 * PS;
  static constexpr int VL = 16 / (int)sizeof(T);                  // values per 16-byte vector
  static constexpr int HC = ((PE + VL - 1) / VL + 1) / 2;         // chunks per row pair
  static constexpr int LDV = 2 * HC * VL + VL;                    // row stride (16-byte multiple)
  static constexpr int VBUF = PE * LDV;
  static constexpr int LDS = PE + 1;                              // odd: conflict-free columns
  static constexpr int PW = (NPM + 31) / 32;                      // warps of the pair role
  static constexpr uint32_t OV = 0;
  static constexpr uint32_t OS = OV + 2u * VBUF * (uint32_t)sizeof(T);
  static constexpr uint32_t OT = (OS + (uint32_t)(PE * LDS) * (uint32_t)sizeof(T) + 15u) & ~15u;
  static constexpr uint32_t OR = OT + 2u * TBUF * (uint32_t)sizeof(T);
  static constexpr uint32_t OL = OR + 2u * NPM * (uint32_t)sizeof(JtRot<T>);
  static constexpr uint32_t OI = (OL + (uint32_t)PE * (uint32_t)sizeof(T) + 3u) & ~3u;   // selected set [PE + 2] int
  static constexpr uint32_t ORED = (OI + (uint32_t)(PE + 2) * 4u + 7u) & ~7u;
  static constexpr size_t bytes(int nt) { return (size_t)ORED + (size_t)(2 * (nt / 32) + 2) * 8; }
  // work items per thread of an NT-thread CTA at the largest order
  static constexpr int items_t(int nt) { return (NPM * (NPM - 1) / 2 + (nt - 32 * PW) - 1) / (nt - 32 * PW); }
  static constexpr int items_c(int nt) { return (NPM * HC + (nt - 32 * PW) - 1) / (nt - 32 * PW); }
  static_assert(8 * PS >= PE * LDS, "the tile region doubles as the product buffer");
  static_assert(LDV >= LDS, "a V buffer holds the transposed eigenvectors with the odd stride");
  static_assert((LDV * sizeof(T)) % 16 == 0 && (VBUF * sizeof(T)) % 16 == 0, "16-byte rows");
};

template <class T>
__device__ __forceinline__ T jt2_ld(const unsigned char* sm, uint32_t off) {
  return *reinterpret_cast<const T*>(sm + off);
}
template <class T>
__device__ __forceinline__ void jt2_st(unsigned char* sm, uint32_t off, T v) {
  *reinterpret_cast<T*>(sm + off) = v;
}

// Per-thread fixed work of the solve (byte offsets into buffer 0; see the
// file comment).  Item threads use t* and c*; pair-role threads reuse the
// first words for their own offsets.
template <int TI, int CI>
struct Jt2Work {
  uint32_t ts[TI], tk[TI], tl[TI], td[TI][4];
  uint32_t cs[CI], ca[CI], cb[CI], cr[CI];
};

// One round at buffer parity PAR (current buffers PAR, next 1 - PAR).
template <class T, int PMAX, int TI, int CI, int PAR>
__device__ __forceinline__ void jt2_round(unsigned char* sm, const Jt2Work<TI, CI>& w, bool items, bool prole,
                                          bool has_next,
                                          uint32_t g_diag, uint32_t g_da, uint32_t g_dab, uint32_t g_db,
                                          uint32_t g_rot, uint32_t g_t, uint32_t g_rk, uint32_t g_rl,
                                          uint32_t g_dk, uint32_t g_dl, uint32_t g_fl, T thresh) {
  using G = Jt2Geo<T, PMAX>;
  using VT = typename Vec16<T>::type;
  constexpr uint32_t TB = sizeof(T);
  constexpr uint32_t CUR_T = PAR * G::TBUF * TB, NXT_T = (1 - PAR) * G::TBUF * TB;
  constexpr uint32_t CUR_R = PAR * G::NPM * sizeof(JtRot<T>), NXT_R = (1 - PAR) * G::NPM * sizeof(JtRot<T>);
  constexpr uint32_t CUR_V = PAR * G::VBUF * TB, NXT_V = (1 - PAR) * G::VBUF * TB;
  constexpr uint32_t P1 = G::PS * TB, P2 = 2 * G::PS * TB, P3 = 3 * G::PS * TB;
  constexpr uint32_t RB = G::LDV * TB, HB = G::HC * G::VL * TB;
  if (items) {
#pragma unroll
    for (int u = 0; u < TI; ++u) {
      if (w.ts[u] == 0xffffffffu) continue;
      const uint32_t s = w.ts[u] + CUR_T;
      const T aa = jt2_ld<T>(sm, s), ab = jt2_ld<T>(sm, s + P1), ba = jt2_ld<T>(sm, s + P2),
              bb = jt2_ld<T>(sm, s + P3);
      const JtRot<T> rk = jt2_ld<JtRot<T>>(sm, w.tk[u] + CUR_R), rl = jt2_ld<JtRot<T>>(sm, w.tl[u] + CUR_R);
      // rows of pair k, then columns of pair l
      const T y00 = jt_cms(rk.c, rk.s, aa, ba), y01 = jt_cms(rk.c, rk.s, ab, bb);
      const T y10 = jt_spc(rk.c, rk.s, aa, ba), y11 = jt_spc(rk.c, rk.s, ab, bb);
      jt2_st<T>(sm, w.td[u][0] + NXT_T, jt_cms(rl.c, rl.s, y00, y01));
      jt2_st<T>(sm, w.td[u][1] + NXT_T, jt_spc(rl.c, rl.s, y00, y01));
      jt2_st<T>(sm, w.td[u][2] + NXT_T, jt_cms(rl.c, rl.s, y10, y11));
      jt2_st<T>(sm, w.td[u][3] + NXT_T, jt_spc(rl.c, rl.s, y10, y11));
    }
#pragma unroll
    for (int u = 0; u < CI; ++u) {
      if (w.cs[u] == 0xffffffffu) continue;
      const uint32_t s = w.cs[u] + CUR_V;
      const JtRot<T> r = jt2_ld<JtRot<T>>(sm, w.cr[u] + CUR_R);
      VT a0 = jt2_ld<VT>(sm, s), a1 = jt2_ld<VT>(sm, s + HB);
      VT b0 = jt2_ld<VT>(sm, s + RB), b1 = jt2_ld<VT>(sm, s + RB + HB);
      jt2_rotv(a0, b0, r);
      jt2_rotv(a1, b1, r);
      jt2_st<VT>(sm, w.ca[u] + NXT_V, a0);
      jt2_st<VT>(sm, w.ca[u] + NXT_V + HB, a1);
      jt2_st<VT>(sm, w.cb[u] + NXT_V, b0);
      jt2_st<VT>(sm, w.cb[u] + NXT_V + HB, b1);
    }
  } else if (prole) {
    // diagonal tile of this pair: the rotation annihilates its coupling
    const uint32_t s = g_diag + CUR_T;
    JtQuad<T> x;
    x.aa = jt2_ld<T>(sm, s); x.ab = jt2_ld<T>(sm, s + P1); x.ba = T(0); x.bb = jt2_ld<T>(sm, s + P3);
    const JtRot<T> r = jt2_ld<JtRot<T>>(sm, g_rot + CUR_R);
    jt2_st<T>(sm, g_da + NXT_T, jt_diag_a(x, r));
    jt2_st<T>(sm, g_dab + NXT_T, r.s != T(0) ? T(0) : x.ab);
    jt2_st<T>(sm, g_db + NXT_T, jt_diag_b(x, r));
    if (has_next) {
      JtRot<T> rn{T(1), T(0)};
      if (!(g_fl & 8u)) {
        const uint32_t q = g_fl & 3u;
        const bool srow = (g_fl & 4u) != 0;
        const uint32_t ts = g_t + CUR_T;
        JtQuad<T> t;
        t.aa = jt2_ld<T>(sm, ts); t.ab = jt2_ld<T>(sm, ts + P1); t.ba = jt2_ld<T>(sm, ts + P2);
        t.bb = jt2_ld<T>(sm, ts + P3);
        const JtRot<T> rk = jt2_ld<JtRot<T>>(sm, g_rk + CUR_R), rl = jt2_ld<JtRot<T>>(sm, g_rl + CUR_R);
        JtQuad<T> dk, dl;
        dk.aa = jt2_ld<T>(sm, g_dk + CUR_T); dk.ab = jt2_ld<T>(sm, g_dk + CUR_T + P1); dk.ba = T(0);
        dk.bb = jt2_ld<T>(sm, g_dk + CUR_T + P3);
        dl.aa = jt2_ld<T>(sm, g_dl + CUR_T); dl.ab = jt2_ld<T>(sm, g_dl + CUR_T + P1); dl.ba = T(0);
        dl.bb = jt2_ld<T>(sm, g_dl + CUR_T + P3);
        // the coupling entry (row i = q >> 1 of pair k, column j = q & 1 of pair l)
        const T y0 = (q >> 1) ? jt_spc(rk.c, rk.s, t.aa, t.ba) : jt_cms(rk.c, rk.s, t.aa, t.ba);
        const T y1 = (q >> 1) ? jt_spc(rk.c, rk.s, t.ab, t.bb) : jt_cms(rk.c, rk.s, t.ab, t.bb);
        const T z = (q & 1) ? jt_spc(rl.c, rl.s, y0, y1) : jt_cms(rl.c, rl.s, y0, y1);
        const T drow = (q >> 1) ? jt_diag_b(dk, rk) : jt_diag_a(dk, rk);
        const T dcol = (q & 1) ? jt_diag_b(dl, rl) : jt_diag_a(dl, rl);
        rn = srow ? jt_rotation(drow, z, dcol, thresh) : jt_rotation(dcol, z, drow, thresh);
      }
      jt2_st<JtRot<T>>(sm, g_rot + NXT_R, rn);
    }
  }
  __syncthreads();
}

// Solve for the block whose round-0 tiles are in tile buffer 0, with the
// eigenvectors by slot in V buffer 0.  Returns the sweeps run (negative if
// max_sweeps was reached first); *par = the buffer holding the result.
// Requires p <= PMAX, TI >= items_t(NT), CI >= items_c(NT).
template <class T, int NT, int PMAX, int TI, int CI>
__device__ __forceinline__ int jt2_solve(unsigned char* sm, int p, double tol, int max_sweeps, int* par_out) {
  using G = Jt2Geo<T, PMAX>;
  constexpr uint32_t TB = sizeof(T), RS = sizeof(JtRot<T>);
  constexpr int IT0 = 32 * G::PW, NIT = NT - IT0;
  static_assert(NIT > 0, "CTA too small for the pair role");
  const int pe = p + (p & 1), np = pe / 2, m = pe - 1;
  const int noff = np * (np - 1) / 2;
  const int nv = (p + G::VL - 1) / G::VL;          // 16-byte vectors per row that carry columns < p
  const int hc = nv < G::HC ? nv : G::HC;          // chunks per pair (first vectors 0 .. hc-1)
  const int nch = np * hc;
  const bool odd = (p & 1) != 0;
  const int tid = threadIdx.x;
  const bool pair = tid < IT0;
  auto tile_el = [&](int s, int t) -> uint32_t {   // plane * PS + tile of slot pair (s, t) next round
    const int a = jt_next_slot(s, np), b = jt_next_slot(t, np);
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return (uint32_t)((2 * (lo & 1) + (hi & 1)) * G::PS + jt_tile(lo >> 1, hi >> 1));
  };
  Jt2Work<TI, CI> w;
  uint32_t g_diag = 0, g_da = 0, g_dab = 0, g_db = 0, g_rot = 0, g_t = 0, g_rk = 0, g_rl = 0, g_dk = 0, g_dl = 0,
           g_fl = 8u;
  if (!pair) {
    const int it = tid - IT0;
#pragma unroll
    for (int u = 0; u < TI; ++u) {
      const int t = it + u * NIT;
      w.ts[u] = w.tk[u] = w.tl[u] = 0xffffffffu;
      w.td[u][0] = w.td[u][1] = w.td[u][2] = w.td[u][3] = 0;
      if (t < noff) {
        // off-diagonal tile number t = l (l - 1) / 2 + k, k < l
        int l = (int)((sqrtf(8.0f * (float)t + 1.0f) + 1.0f) * 0.5f);
        while (l * (l - 1) / 2 > t) --l;
        while ((l + 1) * l / 2 <= t) ++l;
        const int k = t - l * (l - 1) / 2;
        w.ts[u] = G::OT + (uint32_t)jt_tile(k, l) * TB;
        w.tk[u] = G::OR + (uint32_t)k * RS;
        w.tl[u] = G::OR + (uint32_t)l * RS;
        w.td[u][0] = G::OT + tile_el(2 * k, 2 * l) * TB;
        w.td[u][1] = G::OT + tile_el(2 * k, 2 * l + 1) * TB;
        w.td[u][2] = G::OT + tile_el(2 * k + 1, 2 * l) * TB;
        w.td[u][3] = G::OT + tile_el(2 * k + 1, 2 * l + 1) * TB;
      }
    }
#pragma unroll
    for (int u = 0; u < CI; ++u) {
      const int j = (NIT - 1 - it) + u * NIT;     // chunks from the other end of the item threads
      w.cs[u] = 0xffffffffu;
      w.ca[u] = w.cb[u] = w.cr[u] = 0;
      if (j < nch) {
        const int k = j / hc, c = j - k * hc;
        const uint32_t col = (uint32_t)(c * G::VL) * TB;
        w.cs[u] = G::OV + (uint32_t)(2 * k) * G::LDV * TB + col;
        w.ca[u] = G::OV + (uint32_t)jt_next_slot(2 * k, np) * G::LDV * TB + col;
        w.cb[u] = G::OV + (uint32_t)jt_next_slot(2 * k + 1, np) * G::LDV * TB + col;
        w.cr[u] = G::OR + (uint32_t)k * RS;
      }
    }
  } else if (tid < np) {
    const int g = tid;
    g_diag = G::OT + (uint32_t)jt_tile(g, g) * TB;
    g_da = G::OT + tile_el(2 * g, 2 * g) * TB;
    g_dab = G::OT + tile_el(2 * g, 2 * g + 1) * TB;
    g_db = G::OT + tile_el(2 * g + 1, 2 * g + 1) * TB;
    g_rot = G::OR + (uint32_t)g * RS;
    int sg = 0, tg = 0;   // old slots that move to 2g and 2g + 1
    for (int s = 0; s < pe; ++s) {
      const int d = jt_next_slot(s, np);
      if (d == 2 * g) sg = s;
      if (d == 2 * g + 1) tg = s;
    }
    const int ks = sg >> 1, kt = tg >> 1;
    const bool srow = ks < kt;                     // slot sg is the tile's row slot
    const int k = srow ? ks : kt, l = srow ? kt : ks;
    const uint32_t q = srow ? (uint32_t)(((sg & 1) << 1) | (tg & 1)) : (uint32_t)(((tg & 1) << 1) | (sg & 1));
    g_t = G::OT + (uint32_t)jt_tile(k, l) * TB;
    g_rk = G::OR + (uint32_t)k * RS;
    g_rl = G::OR + (uint32_t)l * RS;
    g_dk = G::OT + (uint32_t)jt_tile(k, k) * TB;
    g_dl = G::OT + (uint32_t)jt_tile(l, l) * TB;
    g_fl = q | (srow ? 4u : 0u) | ((odd && g == 0) ? 8u : 0u);
  }
  const bool prole = pair && tid < np;
  double* red = reinterpret_cast<double*>(sm + G::ORED);

  const double tol_eff = fmax(tol, 4.0 * Eps<T>::v * sqrt((double)p));
  const double tol2 = tol_eff * tol_eff;
  constexpr uint32_t P1 = G::PS * TB, P2 = 2 * G::PS * TB, P3 = 3 * G::PS * TB;
  double prev_off2 = 0.0;
  int result = -max_sweeps;
  int par = 0;
  for (int sweep = 0;; ++sweep) {
    // ---- convergence test on the current tiles
    const uint32_t cur = (uint32_t)par * G::TBUF * TB;
    T part[2] = {T(0), T(0)};   // off-diagonal, diagonal sums of squares
    if (!pair) {
#pragma unroll
      for (int u = 0; u < TI; ++u) {
        if (w.ts[u] == 0xffffffffu) continue;
        const uint32_t s = w.ts[u] + cur;
        const T aa = jt2_ld<T>(sm, s), ab = jt2_ld<T>(sm, s + P1), ba = jt2_ld<T>(sm, s + P2),
                bb = jt2_ld<T>(sm, s + P3);
        part[0] += T(2) * (aa * aa + ab * ab + ba * ba + bb * bb);
      }
    } else if (prole) {
      const T aa = jt2_ld<T>(sm, g_diag + cur), ab = jt2_ld<T>(sm, g_diag + cur + P1),
              bb = jt2_ld<T>(sm, g_diag + cur + P3);
      part[0] += T(2) * ab * ab;
      part[1] += aa * aa + bb * bb;
    }
    double sums[2];
    block_sum_t<2, T>(part, sums, red);
    const double off2 = sums[0], tot2 = sums[0] + sums[1];
    if (off2 <= tol2 * tot2 || (sweep >= 5 && off2 > 0.5 * prev_off2)) { result = sweep; break; }
    if (sweep >= max_sweeps) break;
    prev_off2 = off2;
    const T thresh = (T)(tol_eff * sqrt(tot2) / (4.0 * p));
    if (prole) {
      JtRot<T> r{T(1), T(0)};
      if (!(g_fl & 8u)) {
        const T aa = jt2_ld<T>(sm, g_diag + cur), ab = jt2_ld<T>(sm, g_diag + cur + P1),
                bb = jt2_ld<T>(sm, g_diag + cur + P3);
        r = jt_rotation(aa, ab, bb, thresh);
      }
      jt2_st<JtRot<T>>(sm, g_rot + (uint32_t)par * G::NPM * RS, r);
    }
    __syncthreads();
    for (int rd = 0; rd < m; ++rd) {
      const bool nx = rd + 1 < m;
      if (par == 0)
        jt2_round<T, PMAX, TI, CI, 0>(sm, w, !pair, prole, nx, g_diag, g_da, g_dab, g_db, g_rot, g_t, g_rk, g_rl,
                                      g_dk, g_dl, g_fl, thresh);
      else
        jt2_round<T, PMAX, TI, CI, 1>(sm, w, !pair, prole, nx, g_diag, g_da, g_dab, g_db, g_rot, g_t, g_rk, g_rl,
                                      g_dk, g_dl, g_fl, thresh);
      par ^= 1;
    }
  }
  *par_out = par;
  return result;
}

// a7 with jt2_solve: the projection, relaxation input and fused dual update
// of k_psd_fwd_jt, on the geometry of Jt2Geo<T, PMAX> (one CTA per block of
// order p <= PMAX).  Outside the solve the eigenvectors are rows of Vt in
// index order; the solve runs on the slot-ordered copy in the other buffer.
// The projection of block blk by the whole CTA, in the CTA's dynamic shared
// memory (Jt2Geo<T, PMAX>::bytes(NT) of it); shared by the per-step kernel
// below and the persistent forward of kernels_persist.cuh.
template <class T, class V, int NT, int PMAX, int TI, int CI>
__device__ __forceinline__ void jt2_project(const Prob<T, V>& P, const PsdIterIO<T>& io, T* lam_slot, T* U_slot,
                                            double tol, int max_sweeps, int32_t* flags, int blk,
                                            unsigned long long* stats, const T* U_prev) {
  using G = Jt2Geo<T, PMAX>;
  constexpr int ldv = G::LDV, lds = G::LDS;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int p = P.psd_p[blk];
  const int pe = p + (p & 1), np = pe / 2;
  const int64_t row0 = P.psd_row0[blk];
  T* const V0 = reinterpret_cast<T*>(smraw + G::OV);
  T* const V1 = V0 + G::VBUF;
  T* const S = reinterpret_cast<T*>(smraw + G::OS);
  T* const X = reinterpret_cast<T*>(smraw + G::OT);
  T* const lamv = reinterpret_cast<T*>(smraw + G::OL);
  const int inst = io.row_inst[row0];
  const T al = io.alpha[inst], rh = io.rho[row0];
  const int d = p * (p + 1) / 2;
  const bool warm = U_prev != nullptr;
  // index-ordered Vt in buffer 1: identity (cold) or the previous step's
  // eigenvectors as rows; the padding index of odd p keeps its unit vector
  for (int e = threadIdx.x; e < pe * ldv; e += NT) {
    const int i = e / ldv, j = e - i * ldv;
    V1[e] = (i == j && (!warm || i >= p)) ? T(1) : T(0);
  }
  __syncthreads();
  if (warm) {
    const T* Up = U_prev + P.psd_uoff[blk];
    for (int e = threadIdx.x; e < p * p; e += NT) {
      const int j = e / p, i = e - j * p;
      V1[j * ldv + i] = Up[e];
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
    // B = V' S V (upper triangle read below): C = Vt S into X, then C Vt' into S
    jt2_gemm<T>(p, V1, ldv, S, lds, 1, [&](int i, int j, T v) { X[i * lds + j] = v; });
    __syncthreads();
    // (X Vt')(i, j) formed as (Vt X')(j, i): the lanes then walk X with its odd
    // row stride instead of Vt with its 16-byte-multiple one (no bank conflicts)
    jt2_gemm<T>(p, V1, ldv, X, 1, lds, [&](int j, int i, T v) { S[i * lds + j] = v; });
    __syncthreads();
  }
  // round-0 tiles (slot layout, tile buffer 0) from the upper triangle of S,
  // and the eigenvectors by slot into buffer 0
  {
    const int ntri = np * (np + 1) / 2;
    for (int e = threadIdx.x; e < ntri; e += NT) {
      int k, l;
      svec_ij(e, k, l);
      const int a0 = jt_slot_index(0, 2 * k, np), a1 = jt_slot_index(0, 2 * k + 1, np);
      const int b0 = jt_slot_index(0, 2 * l, np), b1 = jt_slot_index(0, 2 * l + 1, np);
      auto at = [&](int i, int j) -> T {
        if (i >= p || j >= p) return T(0);
        return i <= j ? S[i * lds + j] : S[j * lds + i];
      };
      const int E = jt_tile(k, l);
      X[E] = at(a0, b0);
      X[G::PS + E] = at(a0, b1);
      X[2 * G::PS + E] = at(a1, b0);
      X[3 * G::PS + E] = at(a1, b1);
    }
    for (int e = threadIdx.x; e < pe * ldv; e += NT) {
      const int s = e / ldv, j = e - s * ldv;
      V0[e] = V1[jt_slot_index(0, s, np) * ldv + j];
    }
  }
  __syncthreads();
  int par = 0;
  const int sweeps = jt2_solve<T, NT, PMAX, TI, CI>(smraw, p, tol, max_sweeps, &par);
  if (threadIdx.x == 0) {
    if (sweeps < 0) atomicOr(&flags[inst], F_EIG_CAP);
    if (stats) {
      atomicAdd(&stats[0], (unsigned long long)(sweeps < 0 ? -sweeps : sweeps));
      atomicAdd(&stats[1], 1ull);
    }
  }
  // back to index order (every index is in its round-0 slot after whole sweeps)
  T* const Vs = par ? V1 : V0;
  T* const Vt = par ? V0 : V1;
  for (int e = threadIdx.x; e < pe * ldv; e += NT) {
    const int s = e / ldv, j = e - s * ldv;
    Vt[jt_slot_index(0, s, np) * ldv + j] = Vs[e];
  }
  __syncthreads();
  // Vt' with the odd row stride in the free buffer, for Vt Vt' below
  T* const Vtt = Vs;
  for (int e = threadIdx.x; e < p * p; e += NT) {
    const int i = e / p, k = e - i * p;
    Vtt[k * lds + i] = Vt[i * ldv + k];
  }
  __syncthreads();
  // Refinement (as in k_psd_fwd_jt): one Newton-Schulz step on Vt, the
  // Rayleigh-Ritz matrix A = Vt S Vt' of S formed again, eigenvalues
  // L = diag A, and Pi = Vt' (max(L, 0) + G o E) Vt with E the off-diagonal
  // of A and G the Loewner matrix of max(x, 0) at L (Eq. lowner).
  jt2_gemm<T>(p, Vt, ldv, Vtt, lds, 1, [&](int i, int j, T v) { X[i * lds + j] = v; });
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
  jt2_gemm<T>(p, Vt, ldv, S, lds, 1, [&](int i, int j, T v) { X[i * lds + j] = v; });
  __syncthreads();
  // X = Vt S: eigenvalues, the tape, the selected index set, then Pi from
  // the rows of the Rayleigh-Ritz matrix at that set (kernels_jt.cuh)
  int* const sel = reinterpret_cast<int*>(smraw + G::OI);
  jt_rr_diag<T>(p, Vt, ldv, X, lds, lamv);
  __syncthreads();
  jt_select<T>(p, lamv, sel, G::PE);
  T* lam = lam_slot + P.psd_loff[blk];
  T* U = U_slot + P.psd_uoff[blk];
  for (int k = threadIdx.x; k < p; k += NT) lam[k] = lamv[k];
  for (int e = threadIdx.x; e < p * p; e += NT) {
    const int k = e / p, i = e - k * p;
    U[e] = Vt[k * ldv + i];
  }
  __syncthreads();
  const int ns = sel[G::PE];
  const bool usepos = sel[G::PE + 1] != 0;
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

template <class T, class V, int NT, int PMAX, int TI, int CI>
__global__ void __launch_bounds__(NT, 32768 / (NT * 32))
    k_psd_fwd_jt2(Prob<T, V> P, PsdIterIO<T> io, T* lam_slot, T* U_slot, double tol, int max_sweeps,
                  int32_t* flags, int sched_off, unsigned long long* stats, const T* U_prev) {
  jt2_project<T, V, NT, PMAX, TI, CI>(P, io, lam_slot, U_slot, tol, max_sweeps, flags,
                                      P.psd_sched[sched_off + blockIdx.x], stats, U_prev);
}

}  // namespace cosmo
