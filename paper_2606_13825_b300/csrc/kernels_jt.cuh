// Cyclic Jacobi eigensolver for one symmetric block per CTA, with the matrix
// kept in "slot" coordinates (the eigensolver of the PSD projection,
// Sec. 2.4, Eq. psd-proj).
//
// Ordering: the round-robin ("tournament") parallel ordering of Brent & Luk
// (1985).  With pe = p + (p odd) indices and m = pe - 1, round rd pairs
// index m with rd and (rd + k) mod m with (rd - k) mod m, k = 1..pe/2 - 1.
// Slot 2k holds the first index of pair k, slot 2k+1 the second.  From one
// round to the next every index moves to a slot given by a fixed permutation
// pi of the slots (independent of the round; jt_next_slot), and after the m
// rounds of a sweep every index is back in its first slot.
//
// Layout: A is stored by slots, as 2x2 tiles (slots 2k, 2k+1) x (2l, 2l+1),
// upper triangle k <= l only, four values per tile (aa, ab, ba, bb; the ba
// entry of a diagonal tile is unused) kept in four planes of ntri values, so
// that the scattered single-value writes of neighbouring threads land in
// neighbouring words (no bank conflicts).  A round updates every tile by the
// two-sided rotation of its two pairs, J_k' X J_l (Golub & Van Loan,
// Alg. 8.5.1 for the 2x2 Schur rotation), and writes each of the four results
// straight into the position the permutation gives it in the next round, in
// a second tile buffer: its destinations are four fixed addresses each
// thread computes once.
//
// The next round's rotations come out of the same pass: each pair of round
// rd+1 couples two slots that sat in one off-diagonal tile of round rd, so the
// thread owning that tile also re-forms the two new diagonal entries (from
// the old diagonal tiles of its two pairs) and computes the new rotation.
// One CTA barrier per round.  The eigenvectors are accumulated in place by
// index: row i of Vt is column i of V (V <- V J), four components per vector
// access.
#pragma once

#include "common.cuh"

namespace cosmo {

// slot of round rd+1 that receives the index held by slot s in round rd
__host__ __device__ __forceinline__ int jt_next_slot(int s, int np) {
  if (s == 0) return 0;
  if (s == 1) return np >= 2 ? 3 : 1;
  const int k = s >> 1;
  if ((s & 1) == 0) return k == 1 ? 1 : s - 2;
  return k == np - 1 ? 2 * (np - 1) : s + 2;
}

// index held by slot s in round rd (0 <= rd < 2 np - 1)
__host__ __device__ __forceinline__ int jt_slot_index(int rd, int s, int np) {
  const int m = 2 * np - 1, k = s >> 1;
  if (k == 0) return (s & 1) ? rd : m;
  int a = rd + k;
  if (a >= m) a -= m;
  int b = rd - k + m;
  if (b >= m) b -= m;
  return (s & 1) ? b : a;
}

// linear index of tile (k, l), k <= l: column-major upper triangle
__host__ __device__ __forceinline__ int jt_tile(int k, int l) { return l * (l + 1) / 2 + k; }

template <class T> struct __align__(4 * sizeof(T)) JtQuad { T aa, ab, ba, bb; };
template <class T> struct __align__(2 * sizeof(T)) JtRot { T c, s; };

__host__ __device__ inline int jt_ldv(int p) { return (p + 3) & ~3; }
__host__ __device__ inline int jt_lds(int p) { return p | 1; }
__host__ __device__ inline int jt_ntri(int p) {
  const int np = (p + (p & 1)) / 2;
  return np * (np + 1) / 2;
}

// Shared memory of the projection with this solver (bytes).  Layout:
//   Vt  [pe][ldv]   eigenvectors by row (row i = column i of V)
//   S   [p][lds]    the block (and the warm-start products)
//   X   max(p lds, 8 ntri) reals: a product buffer, then the two tile buffers
//   rec [2][np]     rotations (c, s) of the current and the next round
//   sel [p + 2] int, lamv [p] real, red [2 (nt / 32) + 2] double
template <class T>
__host__ __device__ inline size_t jt_smem(int p, int nt) {
  const int pe = p + (p & 1), np = pe / 2;
  const size_t x = (size_t)(p * jt_lds(p) > 8 * jt_ntri(p) ? p * jt_lds(p) : 8 * jt_ntri(p));
  size_t b = (size_t)pe * jt_ldv(p) * sizeof(T);
  b = (b + 31) & ~(size_t)31;
  b += (size_t)p * jt_lds(p) * sizeof(T);
  b = (b + 31) & ~(size_t)31;
  b += x * sizeof(T);
  b = (b + 31) & ~(size_t)31;
  b += (size_t)2 * np * sizeof(JtRot<T>);
  b += (size_t)(p + 2) * sizeof(int);
  b = (b + 15) & ~(size_t)15;
  b += (size_t)p * sizeof(T);
  b = (b + 15) & ~(size_t)15;
  b += (size_t)(2 * (nt / 32) + 2) * sizeof(double);
  return b + 32;
}

template <class T>
struct JtSmem {
  T* Vt; T* S; T* X; JtRot<T>* rec; int* sel; T* lamv; double* red;
  __device__ JtSmem(unsigned char* raw, int p) {
    const int pe = p + (p & 1), np = pe / 2;
    const size_t x = (size_t)(p * jt_lds(p) > 8 * jt_ntri(p) ? p * jt_lds(p) : 8 * jt_ntri(p));
    uintptr_t a = (reinterpret_cast<uintptr_t>(raw) + 31) & ~uintptr_t(31);
    Vt = reinterpret_cast<T*>(a);
    a += (uintptr_t)pe * jt_ldv(p) * sizeof(T);
    a = (a + 31) & ~uintptr_t(31);
    S = reinterpret_cast<T*>(a);
    a += (uintptr_t)p * jt_lds(p) * sizeof(T);
    a = (a + 31) & ~uintptr_t(31);
    X = reinterpret_cast<T*>(a);
    a += x * sizeof(T);
    a = (a + 31) & ~uintptr_t(31);
    rec = reinterpret_cast<JtRot<T>*>(a);
    a += (uintptr_t)2 * np * sizeof(JtRot<T>);
    sel = reinterpret_cast<int*>(a);
    a += (uintptr_t)(p + 2) * sizeof(int);
    a = (a + 15) & ~uintptr_t(15);
    lamv = reinterpret_cast<T*>(a);
    a += (uintptr_t)p * sizeof(T);
    a = (a + 15) & ~uintptr_t(15);
    red = reinterpret_cast<double*>(a);
  }
};

// 2x2 Schur rotation of [[aa, ab], [ab, bb]] (rows: r_a <- c r_a - s r_b,
// r_b <- s r_a + c r_b), skipped (identity) when |ab| <= thresh or when the
// root overflows.  t = sign(theta) phi / (|theta| + sqrt(theta^2 +
// phi^2)) with theta = bb - aa, phi = 2 ab is the smaller root of
// t^2 + 2 (theta/phi) t - 1 = 0.
__device__ __forceinline__ float jt_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double jt_rsqrt(double x) { return rsqrt(x); }

template <class T>
__device__ __forceinline__ JtRot<T> jt_rotation(T aa, T ab, T bb, T thresh) {
  JtRot<T> r{T(1), T(0)};
  if (fabs(ab) > thresh) {
    const T theta = bb - aa, phi = T(2) * ab;
    const T h = hypot(theta, phi);   // scaled: no under/overflow of the squares
    if (h > T(0) && h <= MaxVal<T>::v) {
      const T t = copysign(T(1), theta) * phi / (fabs(theta) + h);
      r.c = jt_rsqrt(fma(t, t, T(1)));
      r.s = t * r.c;
    }
  }
  return r;
}

// FP32: the same rotation from approximate hardware functions on theta, phi
// scaled by max(|theta|, |phi|) (reciprocal and quotient by the fast divide,
// the root as x rsqrt(x); a few ulp each), the IEEE form when that scale is
// outside [1e-30, 1e30].  An inexact t only leaves a small coupling for the
// next sweep; (c, s) stay a rotation to the accuracy of rsqrt (c = rsqrt(1 +
// t^2), s = t c), as in the IEEE form.
template <>
__device__ __forceinline__ JtRot<float> jt_rotation<float>(float aa, float ab, float bb, float thresh) {
  JtRot<float> r{1.0f, 0.0f};
  if (fabsf(ab) > thresh) {
    const float theta = bb - aa, phi = 2.0f * ab;
    const float M = fmaxf(fabsf(theta), fabsf(phi));
    float t;
    if (M >= 1e-30f && M <= 1e30f) {
      const float inv = __fdividef(1.0f, M);
      const float th = theta * inv, ph = phi * inv;   // the larger is +-1
      const float h2 = fmaf(th, th, ph * ph);         // in [1, 2]
      t = copysignf(1.0f, theta) * __fdividef(ph, fmaf(h2, rsqrtf(h2), fabsf(th)));
    } else {
      const float h = hypotf(theta, phi);
      if (!(h > 0.0f && h <= MaxVal<float>::v)) return r;
      t = copysignf(1.0f, theta) * phi / (fabsf(theta) + h);
    }
    r.c = rsqrtf(fmaf(t, t, 1.0f));
    r.s = t * r.c;
  }
  return r;
}

// The rotation's two combinations c a - s b and s a + c b with the rounding
// fixed in the source (the second product rounded, the first fused), so that
// the kernels applying rotations produce the same bits whatever contraction
// the compiler would choose in each context.
template <class T>
__device__ __forceinline__ T jt_cms(T c, T s, T a, T b) { return fma(c, a, -(s * b)); }
template <class T>
__device__ __forceinline__ T jt_spc(T c, T s, T a, T b) { return fma(s, a, c * b); }

// new diagonal entry of a pair's first (second) index after its rotation
template <class T>
__device__ __forceinline__ T jt_diag_a(const JtQuad<T>& q, JtRot<T> r) {
  const T cc = r.c * r.c, cs2 = T(2) * r.c * r.s, ss = r.s * r.s;
  return fma(cc, q.aa, fma(ss, q.bb, -(cs2 * q.ab)));
}
template <class T>
__device__ __forceinline__ T jt_diag_b(const JtQuad<T>& q, JtRot<T> r) {
  const T cc = r.c * r.c, cs2 = T(2) * r.c * r.s, ss = r.s * r.s;
  return fma(ss, q.aa, fma(cc, q.bb, cs2 * q.ab));
}

// Shared-memory accesses by byte offset from the kernel's shared array: with
// the array itself as the base the compiler keeps 32-bit shared addressing.
// tile E of the buffer at byte offset buf (four planes of ntri values)
template <class T>
__device__ __forceinline__ JtQuad<T> jt_ldq(const unsigned char* sm, uint32_t buf, uint32_t E, uint32_t ntri) {
  const T* b = reinterpret_cast<const T*>(sm + buf);
  JtQuad<T> q;
  q.aa = b[E]; q.ab = b[ntri + E]; q.ba = b[2 * ntri + E]; q.bb = b[3 * ntri + E];
  return q;
}
template <class T>
__device__ __forceinline__ JtRot<T> jt_ldr(const unsigned char* sm, uint32_t off) {
  return *reinterpret_cast<const JtRot<T>*>(sm + off);
}
template <class T>
__device__ __forceinline__ void jt_st(unsigned char* sm, uint32_t off, T v) {
  *reinterpret_cast<T*>(sm + off) = v;
}

// rows a, b of Vt (byte offsets ra, rb of the same chunk) <- rotation
template <class T>
__device__ __forceinline__ void jt_rot4(unsigned char* sm, uint32_t ra, uint32_t rb, JtRot<T> r);
template <>
__device__ __forceinline__ void jt_rot4<float>(unsigned char* sm, uint32_t ra, uint32_t rb, JtRot<float> r) {
  float4* pa = reinterpret_cast<float4*>(sm + ra);
  float4* pb = reinterpret_cast<float4*>(sm + rb);
  const float4 x = *pa, y = *pb;
  *pa = make_float4(jt_cms(r.c, r.s, x.x, y.x), jt_cms(r.c, r.s, x.y, y.y), jt_cms(r.c, r.s, x.z, y.z),
                    jt_cms(r.c, r.s, x.w, y.w));
  *pb = make_float4(jt_spc(r.c, r.s, x.x, y.x), jt_spc(r.c, r.s, x.y, y.y), jt_spc(r.c, r.s, x.z, y.z),
                    jt_spc(r.c, r.s, x.w, y.w));
}
template <>
__device__ __forceinline__ void jt_rot4<double>(unsigned char* sm, uint32_t ra, uint32_t rb, JtRot<double> r) {
  double2* pa = reinterpret_cast<double2*>(sm + ra);
  double2* pb = reinterpret_cast<double2*>(sm + rb);
  const double2 x0 = pa[0], x1 = pa[1], y0 = pb[0], y1 = pb[1];
  pa[0] = make_double2(jt_cms(r.c, r.s, x0.x, y0.x), jt_cms(r.c, r.s, x0.y, y0.y));
  pa[1] = make_double2(jt_cms(r.c, r.s, x1.x, y1.x), jt_cms(r.c, r.s, x1.y, y1.y));
  pb[0] = make_double2(jt_spc(r.c, r.s, x0.x, y0.x), jt_spc(r.c, r.s, x0.y, y0.y));
  pb[1] = make_double2(jt_spc(r.c, r.s, x1.x, y1.x), jt_spc(r.c, r.s, x1.y, y1.y));
}

// ---------------------------------------------------------------------------
// End of the refinement shared by the slot-layout kernels.  With X = Vt S (the
// first Rayleigh-Ritz product, Vt orthonormal) the Rayleigh-Ritz matrix is
// B = X Vt', its diagonal the eigenvalues L and its off-diagonal E.  The
// projection Pi = Vt' M Vt with M = max(L, 0) + G o E (G the Loewner matrix of
// max(x, 0), Eq. lowner) has M = 0 between two non-positive indices, so with
// A the smaller of the positive and the non-positive index sets (size ns)
//   Pi = sum_{a in A} v_a w_a' + z_a v_a',
//   w_a = sum_j M_aj v_j,  z_a = sum_{j not in A} M_aj v_j
// (v_j = row j of Vt) when A is the positive set, and Pi = S - (the same with
// D = B - M, which vanishes between two positive indices) when A is the
// non-positive one.  This needs the ns rows of B at A (ns p^2 fused
// multiply-adds) instead of B and two p x p products (3 p^3).
// ---------------------------------------------------------------------------

// L_i = sum_k Vt(i, k) X(i, k): the fused multiply-adds, in the same order,
// that form the diagonal of the full product X Vt'
template <class T>
__device__ __forceinline__ void jt_rr_diag(int p, const T* Vt, int ldv, const T* X, int ldx, T* lamv) {
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    T acc = T(0);
    for (int k = 0; k < p; ++k) acc = fma(Vt[i * ldv + k], X[i * ldx + k], acc);
    lamv[i] = acc;
  }
}

// A in increasing order into sel[0 .. ns), ns into sel[cap], 1 into
// sel[cap + 1] if A is the positive set (warp 0, ballot prefix sums)
template <class T>
__device__ __forceinline__ void jt_select(int p, const T* lamv, int* sel, int cap) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int npos = 0;
    for (int k0 = 0; k0 < p; k0 += 32)
      npos += __popc(__ballot_sync(0xffffffffu, k0 + lane < p && lamv[k0 + lane] > T(0)));
    const bool usepos = npos <= p - npos;
    int c = 0;
    for (int k0 = 0; k0 < p; k0 += 32) {
      const int k = k0 + lane;
      const bool in = k < p && ((lamv[k] > T(0)) == usepos);
      const unsigned b = __ballot_sync(0xffffffffu, in);
      if (in) sel[c + __popc(b & ((1u << lane) - 1u))] = k;
      c += __popc(b);
    }
    if (lane == 0) {
      sel[cap] = c;
      sel[cap + 1] = usepos ? 1 : 0;
    }
  }
}

// rows q < ns of M (A positive) or D = B - M (A non-positive) at A into R,
// then w_q into X rows 0 .. ns and z_q into X rows ns .. 2 ns (X is read
// first, so the CTA barrier in between is the caller's: call the two halves
// with one between them)
template <class T>
__device__ __forceinline__ void jt_lowrank_rows(int p, const T* Vt, int ldv, const T* X, int ldx, T* R, int ldr,
                                                const T* lamv, const int* sel, int ns, bool usepos) {
  for (int idx = threadIdx.x; idx < ns * p; idx += blockDim.x) {
    const int j = idx / ns, q = idx - j * ns, i = sel[q];
    const T li = lamv[i], lj = lamv[j];
    T r;
    if (j == i) {
      r = li;                                   // max(l, 0) on A positive, l - max(l, 0) on A non-positive
    } else {
      T b = T(0);
      for (int k = 0; k < p; ++k) b = fma(Vt[j * ldv + k], X[i * ldx + k], b);
      const bool pi = li > T(0), pj = lj > T(0);
      if (pi == pj) {
        r = b;                                  // G = 1 between positives (M), G = 0 between the others (D)
      } else {
        const T lp = pi ? li : lj, ln = pi ? lj : li;
        r = (usepos ? lp : -ln) / (lp - ln) * b;  // G resp. 1 - G of a mixed pair, no cancellation
      }
    }
    R[q * ldr + j] = r;
  }
}
template <class T>
__device__ __forceinline__ void jt_lowrank_wz(int p, const T* Vt, int ldv, T* X, int ldx, const T* R, int ldr,
                                              const T* lamv, int ns, bool usepos) {
  for (int idx = threadIdx.x; idx < ns * p; idx += blockDim.x) {
    const int q = idx / p, c = idx - q * p;
    T w = T(0), z = T(0);
    for (int j = 0; j < p; ++j) {
      const T m = R[q * ldr + j], v = Vt[j * ldv + c];
      w = fma(m, v, w);
      if ((lamv[j] > T(0)) != usepos) z = fma(m, v, z);
    }
    X[q * ldx + c] = w;
    X[(ns + q) * ldx + c] = z;
  }
}
// Pi(i, j) from w, z; sij = S(i, j) (used when A is the non-positive set)
template <class T>
__device__ __forceinline__ T jt_lowrank_entry(int i, int j, const T* Vt, int ldv, const T* X, int ldx,
                                              const int* sel, int ns, bool usepos, T sij) {
  T acc = T(0);
  for (int q = 0; q < ns; ++q) {
    const int a = sel[q];
    acc = fma(Vt[a * ldv + i], X[q * ldx + j], acc);
    acc = fma(X[(ns + q) * ldx + i], Vt[a * ldv + j], acc);
  }
  return usepos ? acc : sij - acc;
}

// items of a round per thread for a CTA of nt threads: the off-diagonal
// tiles and the four-component chunks of the eigenvector rotation
__host__ __device__ inline int jt_items(int p) {
  const int np = (p + (p & 1)) / 2;
  return np * (np - 1) / 2 + np * (jt_ldv(p) / 4);
}
// warps of the pair role (diagonal tiles and next round's rotations); the
// item pool goes to the other threads of the CTA
__host__ __device__ inline int jt_pair_warps(int p) { return ((p + (p & 1)) / 2 + 31) / 32; }
__host__ __device__ inline int jt_ipt(int p, int nt) {
  const int it = nt - 32 * jt_pair_warps(p);
  return it > 0 ? (jt_items(p) + it - 1) / it : 1 << 20;
}

// Solve for the block held in the tile buffer at byte offset tb0 (round-0
// slot layout, padding index zero), accumulating the rotations into Vt
// (identity or a warm start; byte offset vt).  Returns the sweeps run
// (negative if max_sweeps was reached first) and *fin = the byte offset of
// the tile buffer holding the result.  Stops when off(A) <= tol' ||A||_F
// with tol' = max(tol, 4 eps sqrt(p)), or when from the fifth sweep on a
// sweep fails to halve off(A)^2 (the rounding floor); rotations with |a_pq|
// <= tol' ||A||_F / (4p) are skipped (if every coupling is that small,
// off(A) <= tol' ||A||_F / 4 already).
//
// Work of a round: the first np threads (the pair warps) update the diagonal
// tile of their pair and form the rotation of next round's pair of the same
// number from the old tiles (no dependence on this round's writes); every
// thread after the pair warps takes up to IPT items of one pool (off-diagonal
// tiles, then eigenvector chunks).  Requires jt_ipt(p, NT) <= IPT and
// p <= 180.
template <class T, int NT, int IPT>
__device__ __forceinline__ int jt_solve(unsigned char* sm, uint32_t tb0, uint32_t tb1, uint32_t vt,
                                        uint32_t recb, double* red, int p, double tol, int max_sweeps,
                                        uint32_t* fin) {
  constexpr uint32_t RB = sizeof(JtRot<T>), TB = sizeof(T);
  const int pe = p + (p & 1), np = pe / 2, m = pe - 1;
  const int ldv = jt_ldv(p), p4 = ldv / 4;
  const uint32_t VB = (uint32_t)ldv * TB;
  const int noff = np * (np - 1) / 2, nitems = noff + np * p4, ntri = np * (np + 1) / 2;
  const uint32_t nt_ = (uint32_t)ntri;
  const bool odd = (p & 1) != 0;   // pair 0 holds the padding index
  const int tid = threadIdx.x;
  auto dst_of = [&](int s, int t) -> uint32_t {   // element offset of slot pair (s, t) next round
    const int a = jt_next_slot(s, np), b = jt_next_slot(t, np);
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return (uint32_t)((2 * (lo & 1) + (hi & 1)) * ntri + jt_tile(lo >> 1, hi >> 1));
  };
  // ---- items: tile (kind 1): d0 = E | k << 12 | l << 20 | 1 << 28, d1/d2 = destinations;
  //             chunk (kind 2): d0 = c4 | k << 12 | 2 << 28, d1/d2 = current row indices a, b
  uint32_t d0[IPT], d1[IPT], d2[IPT];
  const int it0 = 32 * jt_pair_warps(p), nit = NT - it0;
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const int it = tid >= it0 ? tid - it0 + u * nit : nitems;
    d0[u] = d1[u] = d2[u] = 0;
    if (it < noff) {
      // off-diagonal tile number it = l (l - 1) / 2 + k, k < l
      int l = (int)((sqrtf(8.0f * (float)it + 1.0f) + 1.0f) * 0.5f);
      while (l * (l - 1) / 2 > it) --l;
      while ((l + 1) * l / 2 <= it) ++l;
      const int k = it - l * (l - 1) / 2;
      d0[u] = (uint32_t)jt_tile(k, l) | ((uint32_t)k << 12) | ((uint32_t)l << 20) | (1u << 28);
      d1[u] = dst_of(2 * k, 2 * l) | (dst_of(2 * k, 2 * l + 1) << 16);
      d2[u] = dst_of(2 * k + 1, 2 * l) | (dst_of(2 * k + 1, 2 * l + 1) << 16);
    } else if (it < nitems) {
      const int w = it - noff, k = w / p4, c4 = w - k * p4;
      d0[u] = (uint32_t)c4 | ((uint32_t)k << 12) | (2u << 28);
      d1[u] = (uint32_t)jt_slot_index(0, 2 * k, np);
      d2[u] = (uint32_t)jt_slot_index(0, 2 * k + 1, np);
    }
  }
  // ---- pair role (tid < np): diagonal tile tid, and the rotation of next
  // round's pair tid from the old tile coupling its two slots
  uint32_t g0 = 0, g1 = 0, g2 = 0;
  if (tid < np) {
    const int g = tid;
    g0 = dst_of(2 * g, 2 * g) | (dst_of(2 * g, 2 * g + 1) << 16);
    g1 = dst_of(2 * g + 1, 2 * g + 1) | ((uint32_t)jt_tile(g, g) << 16);
    int sg = 0, tg = 0;   // old slots that move to 2g and 2g + 1
    for (int s = 0; s < pe; ++s) {
      const int d = jt_next_slot(s, np);
      if (d == 2 * g) sg = s;
      if (d == 2 * g + 1) tg = s;
    }
    const int ks = sg >> 1, kt = tg >> 1;
    const bool srow = ks < kt;                 // slot sg is the tile's row slot
    const int k = srow ? ks : kt, l = srow ? kt : ks;
    const int q = srow ? (((sg & 1) << 1) | (tg & 1)) : (((tg & 1) << 1) | (sg & 1));
    g2 = (uint32_t)jt_tile(k, l) | ((uint32_t)k << 12) | ((uint32_t)l << 20) | ((uint32_t)q << 28) |
         ((uint32_t)srow << 30) | ((odd && g == 0) ? (1u << 31) : 0u);
  }

  const double tol_eff = fmax(tol, 4.0 * Eps<T>::v * sqrt((double)p));
  const double tol2 = tol_eff * tol_eff;
  double prev_off2 = 0.0;
  int result = -max_sweeps;
  uint32_t cur = tb0, nxt = tb1;
  int rb = 0;   // rotation buffer of the coming round
  for (int sweep = 0;; ++sweep) {
    // ---- convergence test on the current tiles
    T part[2] = {T(0), T(0)};   // off-diagonal, diagonal sums of squares
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      if ((d0[u] >> 28) != 1) continue;
      const JtQuad<T> x = jt_ldq<T>(sm, cur, d0[u] & 0xfffu, nt_);
      part[0] += T(2) * (x.aa * x.aa + x.ab * x.ab + x.ba * x.ba + x.bb * x.bb);
    }
    if (tid < np) {
      const JtQuad<T> x = jt_ldq<T>(sm, cur, g1 >> 16, nt_);
      part[0] += T(2) * x.ab * x.ab;
      part[1] += x.aa * x.aa + x.bb * x.bb;
    }
    double sums[2];
    block_sum_t<2, T>(part, sums, red);
    const double off2 = sums[0], tot2 = sums[0] + sums[1];
    if (off2 <= tol2 * tot2 || (sweep >= 5 && off2 > 0.5 * prev_off2)) { result = sweep; break; }
    if (sweep >= max_sweeps) break;
    prev_off2 = off2;
    const T thresh = (T)(tol_eff * sqrt(tot2) / (4.0 * p));
    if (tid < np) {
      JtRot<T> r{T(1), T(0)};
      if (!(odd && tid == 0)) {
        const JtQuad<T> x = jt_ldq<T>(sm, cur, g1 >> 16, nt_);
        r = jt_rotation(x.aa, x.ab, x.bb, thresh);
      }
      *reinterpret_cast<JtRot<T>*>(sm + recb + (uint32_t)(rb * np + tid) * RB) = r;
    }
    __syncthreads();
    for (int rd = 0; rd < m; ++rd) {
      const uint32_t rc = recb + (uint32_t)(rb * np) * RB;
      const uint32_t rn = recb + (uint32_t)((rb ^ 1) * np) * RB;
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        const uint32_t kind = d0[u] >> 28;
        if (kind == 1) {
          const uint32_t k = (d0[u] >> 12) & 0xffu, l = (d0[u] >> 20) & 0xffu;
          const JtQuad<T> x = jt_ldq<T>(sm, cur, d0[u] & 0xfffu, nt_);
          const JtRot<T> rk = jt_ldr<T>(sm, rc + k * RB), rl = jt_ldr<T>(sm, rc + l * RB);
          // rows of pair k, then columns of pair l
          const T y00 = jt_cms(rk.c, rk.s, x.aa, x.ba), y01 = jt_cms(rk.c, rk.s, x.ab, x.bb);
          const T y10 = jt_spc(rk.c, rk.s, x.aa, x.ba), y11 = jt_spc(rk.c, rk.s, x.ab, x.bb);
          jt_st<T>(sm, nxt + (d1[u] & 0xffffu) * TB, jt_cms(rl.c, rl.s, y00, y01));
          jt_st<T>(sm, nxt + (d1[u] >> 16) * TB, jt_spc(rl.c, rl.s, y00, y01));
          jt_st<T>(sm, nxt + (d2[u] & 0xffffu) * TB, jt_cms(rl.c, rl.s, y10, y11));
          jt_st<T>(sm, nxt + (d2[u] >> 16) * TB, jt_spc(rl.c, rl.s, y10, y11));
        } else if (kind == 2) {
          const uint32_t k = (d0[u] >> 12) & 0xffu, c4 = d0[u] & 0xfffu;
          const int a = (int)d1[u], b = (int)d2[u];
          const JtRot<T> r = jt_ldr<T>(sm, rc + k * RB);
          if (r.s != T(0) && a < p && b < p)
            jt_rot4<T>(sm, vt + (uint32_t)a * VB + c4 * 4 * TB, vt + (uint32_t)b * VB + c4 * 4 * TB, r);
          // next round's indices of pair k: +1 mod m (the fixed index m of pair 0 stays)
          if (k != 0) d1[u] = a + 1 == m ? 0u : (uint32_t)(a + 1);
          d2[u] = b + 1 == m ? 0u : (uint32_t)(b + 1);
        }
      }
      if (tid < np) {
        // diagonal tile of pair tid: the rotation annihilates its coupling
        const JtQuad<T> x = jt_ldq<T>(sm, cur, g1 >> 16, nt_);
        const JtRot<T> r = jt_ldr<T>(sm, rc + (uint32_t)tid * RB);
        jt_st<T>(sm, nxt + (g0 & 0xffffu) * TB, jt_diag_a(x, r));
        jt_st<T>(sm, nxt + (g0 >> 16) * TB, r.s != T(0) ? T(0) : x.ab);
        jt_st<T>(sm, nxt + (g1 & 0xffffu) * TB, jt_diag_b(x, r));
        if (rd + 1 < m) {
          JtRot<T> rn_{T(1), T(0)};
          if (!(g2 >> 31)) {
            const uint32_t k = (g2 >> 12) & 0xffu, l = (g2 >> 20) & 0xffu, q = (g2 >> 28) & 3u;
            const bool srow = (g2 >> 30) & 1u;
            const JtQuad<T> t = jt_ldq<T>(sm, cur, g2 & 0xfffu, nt_);
            const JtRot<T> rk = jt_ldr<T>(sm, rc + k * RB), rl = jt_ldr<T>(sm, rc + l * RB);
            const JtQuad<T> dk = jt_ldq<T>(sm, cur, (uint32_t)jt_tile(k, k), nt_);
            const JtQuad<T> dl = jt_ldq<T>(sm, cur, (uint32_t)jt_tile(l, l), nt_);
            // the coupling entry (row i = q >> 1 of pair k, column j = q & 1 of pair l)
            const T y0 = (q >> 1) ? jt_spc(rk.c, rk.s, t.aa, t.ba) : jt_cms(rk.c, rk.s, t.aa, t.ba);
            const T y1 = (q >> 1) ? jt_spc(rk.c, rk.s, t.ab, t.bb) : jt_cms(rk.c, rk.s, t.ab, t.bb);
            const T z = (q & 1) ? jt_spc(rl.c, rl.s, y0, y1) : jt_cms(rl.c, rl.s, y0, y1);
            // new diagonal entries of the row slot and of the column slot
            const T drow = (q >> 1) ? jt_diag_b(dk, rk) : jt_diag_a(dk, rk);
            const T dcol = (q & 1) ? jt_diag_b(dl, rl) : jt_diag_a(dl, rl);
            rn_ = srow ? jt_rotation(drow, z, dcol, thresh) : jt_rotation(dcol, z, drow, thresh);
          }
          *reinterpret_cast<JtRot<T>*>(sm + rn + (uint32_t)tid * RB) = rn_;
        }
      }
      __syncthreads();
      const uint32_t t = cur; cur = nxt; nxt = t;
      rb ^= 1;
    }
  }
  *fin = cur;
  return result;
}

}  // namespace cosmo
