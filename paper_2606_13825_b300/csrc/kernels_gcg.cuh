// Grid-wide Jacobi-preconditioned CG for large instances of the reduced
// system (P + sigma I + A'D(rho)A) x = rhs (Sec. 2.3), where one CTA per
// instance cannot reach HBM bandwidth.  Instances are cut into tiles of
// consecutive columns (and rows); every tile is one CTA.  Iteration `it`:
//
//   rows:    t = rho o (A p^),  p^ = z + beta p,  z = D^-1 r  (p^ formed on the fly)
//   cols:    u = sigma p^ + P p^ + A' t,  partial p^'u per tile
//   update:  alpha = r'z / p^'u,  x += alpha p^,  r -= alpha u,  z = D^-1 r,
//            p <- p^,  partials r'z and r'r per tile
//
// z and p are stored interleaved (zp[j] = (z_j, p_j)) so that every gather of
// p^ is one load.  The per-instance scalars (alpha, beta, r'z and the
// stop/continue state) are formed once per kernel by the last tile of the
// instance to finish (an atomic tile counter), which sums the per-tile
// partials in tile order in double: the result does not depend on which tile
// comes last or on scheduling.  Scalars read by the next iteration are double
// buffered by iteration parity.  Zero start only.
#pragma once

#include <cuda/atomic>
#include <type_traits>

#include "common.cuh"

namespace cosmo {

constexpr int GCG_NT = 256;     // threads of every grid-CG CTA
// nonzeros per lane per batch (fits 64 registers without spills)
template <class T> __host__ __device__ constexpr int gcg_u() { return sizeof(T) == 4 ? 8 : 4; }

template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

struct GcgTiles {
  int32_t nct;              // column tiles
  const int32_t* ct_inst;   // [nct]
  const int64_t* ct_lo;     // [nct] first column
  const int64_t* ct_hi;     // [nct] one past the last column
  const int32_t* it_lo;     // [ninst] first column tile of the instance
  const int32_t* it_hi;     // [ninst] one past its last column tile
  int32_t nrt;              // row tiles
  const int32_t* rt_inst;
  const int64_t* rt_lo;
  const int64_t* rt_hi;
  const int32_t* rt_first;  // [nrt] 1 for the first row tile of its instance
  // batch width of the row routine for A, A' and P (gcg_rows_any) and the
  // entry counts of A and P (array ends for the 16-byte loads)
  int32_t vq_a, vq_at, vq_p;
  int64_t nnz_a, nnz_p;
};

template <class T>
struct GcgState {
  using T2 = typename Vec2<T>::type;
  const T* rhs; T* x; const T* rho; const T* dinv; double sigma;
  T* r; T2* zp; T* u; T* t;
  double* part_a;           // [nct] per-tile partials (p^'u, then r'z)
  double* part_b;           // [nct] (r'r)
  int32_t* cnt_grp;         // [nct] tiles of a 32-tile group done in the current kernel
  int32_t* cnt_inst;        // [ninst] groups of the instance done (both 0 between kernels)
  double* sc_rz;            // [2][ninst] r'z at the start of iteration it (parity it & 1)
  double* sc_beta;          // [2][ninst]
  int32_t* sc_state;        // [2][ninst] 0 iterate, 1 converged, 2 cap reached
  double* sc_alpha;         // [ninst]
  double* sc_bb;            // [ninst] ||rhs||^2
  int32_t* iters;           // [ninst] (may be null)
  int32_t* running;         // [maxit + 1] instances still iterating at each iteration
  double tol;
  int32_t maxit;
};

// Called by every thread of a tile after thread 0 stored the tile's partials:
// true in the one tile of the instance that finished last.  Two levels of
// counters (groups of 32 tiles, then the instance) so that no more than 32
// atomics queue on one address; each last arrival resets its counter for
// the next kernel.  cnt_grp is indexed by the group's first tile.  The
// increments are acquire-release read-modify-writes: they publish thread 0's
// partials and, in the last arrival, make every earlier tile's visible (the
// CTA barrier then extends that to the other threads).  A full fence here
// stalls for microseconds while other CTAs stream from HBM.
__device__ __forceinline__ bool gcg_last_tile(int32_t* cnt_grp, int32_t* cnt_inst, int inst, int tile,
                                              int tlo, int thi) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    const int g0 = tlo + ((tile - tlo) & ~31);
    const int gsize = min(32, thi - g0);
    const int ngroups = (thi - tlo + 31) >> 5;
    int last = 0;
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> cg(cnt_grp[g0]);
    if (cg.fetch_add(1, cuda::memory_order_acq_rel) == gsize - 1) {
      cg.store(0, cuda::memory_order_relaxed);
      cuda::atomic_ref<int32_t, cuda::thread_scope_device> ci(cnt_inst[inst]);
      if (ci.fetch_add(1, cuda::memory_order_acq_rel) == ngroups - 1) {
        ci.store(0, cuda::memory_order_relaxed);
        last = 1;
      }
    }
    s_last = last;
  }
  __syncthreads();
  return s_last != 0;
}

// Sum of the instance's per-tile partials in tile order (fixed, whichever tile
// runs it); broadcast to every thread.
template <int NT, int NV>
__device__ __forceinline__ void gcg_tile_sum(double* const (&part)[NV], int lo, int hi, double (&out)[NV],
                                             double* sm) {
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = 0.0;
    for (int k = lo + threadIdx.x; k < hi; k += NT) s += __ldcg(part[q] + k);
    out[q] = s;
  }
  block_sum<NV>(out, sm);
}

__device__ __forceinline__ int gcg_next_state(double rr, double bb, double tol, int it_next, int maxit) {
  if (rr <= tol * tol * bb || !(rr == rr)) return 1;
  return it_next >= maxit ? 2 : 0;
}

// zero start: x = 0, r = rhs, z = D^-1 rhs, p = 0; scalars of iteration 0
template <class T, int NT = GCG_NT>
__global__ void __launch_bounds__(NT) k_gcg_init(GcgTiles G, GcgState<T> S) {
  __shared__ double sm[2 * (NT / 32)];
  const int tile = blockIdx.x;
  const int inst = G.ct_inst[tile];
  T a0 = T(0), a1 = T(0);
  for (int64_t j = G.ct_lo[tile] + threadIdx.x; j < G.ct_hi[tile]; j += NT) {
    const T b = S.rhs[j];
    const T z = S.dinv[j] * b;
    typename Vec2<T>::type g;
    g.x = z;
    g.y = T(0);
    S.x[j] = T(0);
    S.r[j] = b;
    S.zp[j] = g;
    a0 += b * z;
    a1 += b * b;
  }
  const T tv[2] = {a0, a1};
  double acc[2];
  block_sum_t<2>(tv, acc, sm);
  if (threadIdx.x == 0) {
    S.part_a[tile] = acc[0];
    S.part_b[tile] = acc[1];
  }
  const int lo = G.it_lo[inst], hi = G.it_hi[inst];
  if (!gcg_last_tile(S.cnt_grp, S.cnt_inst, inst, tile, lo, hi)) return;
  double* const parts[2] = {S.part_a, S.part_b};
  double tot[2];
  gcg_tile_sum<NT, 2>(parts, lo, hi, tot, sm);
  if (threadIdx.x == 0) {
    S.sc_rz[inst] = tot[0];
    S.sc_beta[inst] = 0.0;
    S.sc_bb[inst] = tot[1];
    S.sc_state[inst] = gcg_next_state(tot[1], tot[1], S.tol, 0, S.maxit);
  }
}

// U nonzeros per lane of one CSR batch: entries k = lane + 32 q < rem of
// (cp, vp); entries past rem read as column -1 with value 0 (every gather
// returns 0 for column -1).
template <int U, class T>
__device__ __forceinline__ void gcg_load_batch(const int32_t* __restrict__ cp, const T* __restrict__ vp, int rem,
                                               int32_t (&c)[U], T (&v)[U]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < U; ++q) {
    const int k = lane + 32 * q;
    const bool ok = k < rem;
    c[q] = ok ? __ldg(cp + k) : -1;
    v[q] = ok ? __ldg(vp + k) : T(0);
  }
}

// One warp over the CSR rows r, r + step, ... < r_end: emit(row, side, sum)
// with sum = sum_e val[e] * gather(col[e]) (in T, fixed order) and side =
// side(row) loaded ahead.  Software pipelined: the next batch of column
// indices and values, the extent of the following row and its side value are
// loaded before the current batch is gathered, so every warp keeps HBM loads
// in flight while it waits on its gathers.
template <int U, class T, class Side, class Gather, class Emit>
__device__ __forceinline__ void gcg_warp_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                              const T* __restrict__ val, int64_t r, int64_t r_end,
                                              int64_t step, Side side, Gather gather, Emit emit) {
  if (r >= r_end) return;
  constexpr int B = 32 * U;
  int64_t e = __ldg(rp + r), e1 = __ldg(rp + r + 1);
  auto sv = side(r);
  int64_t nr = r + step;
  int64_t f0 = 0, f1 = 0;
  decltype(sv) fsv = sv;
  if (nr < r_end) {
    f0 = __ldg(rp + nr);
    f1 = __ldg(rp + nr + 1);
    fsv = side(nr);
  }
  int32_t c[U];
  T v[U];
  gcg_load_batch<U>(ci + e, val + e, (int)min(e1 - e, (int64_t)B), c, v);
  T acc = T(0);
  while (true) {
    const bool row_done = e1 - e <= B;
    const bool more = !row_done || nr < r_end;
    const int64_t ne = row_done ? f0 : e + B;
    const int64_t ne1 = row_done ? f1 : e1;
    int32_t c2[U];
    T v2[U];
    if (more) gcg_load_batch<U>(ci + ne, val + ne, (int)min(ne1 - ne, (int64_t)B), c2, v2);
    const auto cur_sv = sv;
    if (row_done && more) {
      sv = fsv;
      const int64_t nn = nr + step;
      if (nn < r_end) {
        f0 = __ldg(rp + nn);
        f1 = __ldg(rp + nn + 1);
        fsv = side(nn);
      }
    }
#pragma unroll
    for (int q = 0; q < U; ++q) acc += v[q] * gather(c[q]);
    if (row_done) {
      emit(r, cur_sv, warp_allsum(acc));
      acc = T(0);
      r = nr;
      nr += step;
    }
    if (!more) break;
#pragma unroll
    for (int q = 0; q < U; ++q) {
      c[q] = c2[q];
      v[q] = v2[q];
    }
    e = ne;
    e1 = ne1;
  }
}

// 16-byte loads of 4 consecutive entries (column indices and values).
template <class T> struct Vec4Load;
template <> struct Vec4Load<float> {
  static __device__ __forceinline__ void ld(const float* p, float (&x)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
};
template <> struct Vec4Load<double> {
  static __device__ __forceinline__ void ld(const double* p, double (&x)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  }
};

// One warp over the rows r, r + step, ... < r_end, as gcg_warp_rows, the
// entries of a row being [e0, e1) from ext(row, e0, e1), with 16-byte loads:
// lane l takes the 4-entry groups l, l + 32, ... (VQ of them per batch)
// counted from the row start rounded down to a multiple of 4, in
// 32-bit offsets from there.  Entries outside the row read as column -1 with
// value 0 (masked only in the row's first and last groups); lanes past the
// row end load nothing.  Needs ci and val 16-byte aligned; a group that would
// read past nnz (the array end) falls back to single loads.
template <int VQ, class T, class Ext, class Side, class Gather, class Emit>
__device__ __forceinline__ void gcg_warp_rows_ext(Ext ext, const int32_t* __restrict__ ci,
                                                  const T* __restrict__ val, int64_t nnz, int64_t r,
                                                  int64_t r_end, int64_t step, Side side, Gather gather,
                                                  Emit emit) {
  const int lane = threadIdx.x & 31;
  for (; r < r_end; r += step) {
    int64_t e0, e1;
    ext(r, e0, e1);
    const auto sv = side(r);
    const int64_t base = e0 & ~(int64_t)3;
    const int32_t* __restrict__ cb = ci + base;
    const T* __restrict__ xb = val + base;
    const int skip = (int)(e0 - base);                          // 0..3 entries before the row
    const int len = (int)(e1 - base);                           // offset of the row end
    const int lim = (int)min(nnz - base, (int64_t)len + 4);     // readable entries from base
    T acc = T(0);
    for (int off0 = 0; off0 < len; off0 += 128 * VQ) {
      int32_t c[VQ][4];
      T x[VQ][4];
#pragma unroll
      for (int q = 0; q < VQ; ++q) {
        const int og = off0 + 4 * (lane + 32 * q);
        if (og < len) {
          if (og + 4 <= lim) {
            const int4 cv = __ldg(reinterpret_cast<const int4*>(cb + og));
            c[q][0] = cv.x; c[q][1] = cv.y; c[q][2] = cv.z; c[q][3] = cv.w;
            Vec4Load<T>::ld(xb + og, x[q]);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const bool ok = og + k < lim;
              c[q][k] = ok ? __ldg(cb + og + k) : -1;
              x[q][k] = ok ? __ldg(xb + og + k) : T(0);
            }
          }
          if (og < skip || og + 4 > len) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (og + k < skip || og + k >= len) {
                c[q][k] = -1;
                x[q][k] = T(0);
              }
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            c[q][k] = -1;
            x[q][k] = T(0);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < VQ; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc += x[q][k] * gather(c[q][k]);
    }
    emit(r, sv, warp_allsum(acc));
  }
}

// The entries of row r are [rp[r], rp[r + 1]).
template <int VQ, class T, class Side, class Gather, class Emit>
__device__ __forceinline__ void gcg_warp_rows_vec(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                  const T* __restrict__ val, int64_t nnz, int64_t r,
                                                  int64_t r_end, int64_t step, Side side, Gather gather,
                                                  Emit emit) {
  gcg_warp_rows_ext<VQ>([&](int64_t row, int64_t& e0, int64_t& e1) {
    e0 = __ldg(rp + row);
    e1 = __ldg(rp + row + 1);
  }, ci, val, nnz, r, r_end, step, side, gather, emit);
}

// Runs the row routine with the batch width `vq` chosen on the host from the
// matrix's mean row length (1, 2 or 4 groups of 4 per lane, 2 at most for
// double values; 0 = scalar loads when the arrays are not 16-byte aligned).
template <class T, class Side, class Gather, class Emit>
__device__ __forceinline__ void gcg_rows_any(int vq, const int64_t* rp, const int32_t* ci, const T* val,
                                             int64_t nnz, int64_t r, int64_t r_end, int64_t step, Side side,
                                             Gather gather, Emit emit) {
  // double values: at most 2 groups per lane (4 would spill)
  if constexpr (sizeof(T) == 4) {
    if (vq == 4) {
      gcg_warp_rows_vec<4>(rp, ci, val, nnz, r, r_end, step, side, gather, emit);
      return;
    }
  }
  if (vq >= 2) gcg_warp_rows_vec<2>(rp, ci, val, nnz, r, r_end, step, side, gather, emit);
  else if (vq == 1) gcg_warp_rows_vec<1>(rp, ci, val, nnz, r, r_end, step, side, gather, emit);
  else gcg_warp_rows<gcg_u<T>()>(rp, ci, val, r, r_end, step, side, gather, emit);
}

// sP[j - lo] = (P p^)_j for the tile's columns.  Rows of at most 16 entries
// (short = 1; a diagonal P has one) take one thread per row, longer ones one
// warp per row.  Ends with a CTA barrier.
template <int VP = 0, class T, class PHat>
__device__ __forceinline__ void gcg_p_part(const Prob<T, T>& P, const GcgTiles& G, int64_t lo, int64_t hi,
                                           int short_rows,
                                           PHat phat, T* sP) {
  const int nt = blockDim.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (!P.P_rp) {
    for (int64_t j = lo + threadIdx.x; j < hi; j += nt) sP[j - lo] = T(0);
  } else if (short_rows) {
    for (int64_t j = lo + threadIdx.x; j < hi; j += nt) {
      T s = T(0);
      const int64_t e1 = __ldg(P.P_rp + j + 1);
      for (int64_t e = __ldg(P.P_rp + j); e < e1; ++e) s += __ldg(P.P_v + e) * phat(__ldg(P.P_ci + e));
      sP[j - lo] = s;
    }
  } else {
    auto emit = [&](int64_t j, int, T sum) { if (lane == 0) sP[j - lo] = sum; };
    if constexpr (VP > 0)
      gcg_warp_rows_vec<VP>(P.P_rp, P.P_ci, P.P_v, G.nnz_p, lo + w, hi, nt / 32, [&](int64_t) { return 0; }, phat,
                            emit);
    else
      gcg_rows_any(G.vq_p, P.P_rp, P.P_ci, P.P_v, G.nnz_p, lo + w, hi, nt / 32, [&](int64_t) { return 0; }, phat,
                   emit);
  }
  __syncthreads();
}

// rows: t = rho o (A p^); one warp per row.  The first row tile of each
// instance records convergence (iteration count) and counts the instances
// still iterating.
template <class T>
__global__ void __launch_bounds__(GCG_NT, 4) k_gcg_rows(Prob<T, T> P, GcgTiles G, GcgState<T> S, int it) {
  using T2 = typename Vec2<T>::type;
  const int tile = blockIdx.x;
  const int inst = G.rt_inst[tile];
  const int par = it & 1;
  const int st = S.sc_state[par * P.ninst + inst];
  if (G.rt_first[tile] && threadIdx.x == 0) {
    // the state of iteration it - 1 is still in the other parity
    if (st == 0) atomicAdd(&S.running[it], 1);
    else if (S.iters && (it == 0 || S.sc_state[(par ^ 1) * P.ninst + inst] == 0)) S.iters[inst] = it;
  }
  if (st) return;
  const T beta = (T)S.sc_beta[par * P.ninst + inst];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const T2* __restrict__ zp = S.zp;
  const T* __restrict__ rho = S.rho;
  T* __restrict__ t = S.t;
  gcg_rows_any(
      G.vq_a, P.A_rp, P.A_ci, P.A_v, G.nnz_a, G.rt_lo[tile] + w, G.rt_hi[tile], GCG_NT / 32,
      [&](int64_t r) { return __ldg(rho + r); },
      [&](int32_t c) {
        if (c < 0) return T(0);
        const T2 g = __ldg(zp + c);
        return g.x + beta * g.y;
      },
      [&](int64_t r, T rr, T sum) { if (lane == 0) t[r] = rr * sum; });
}

// cols: u = sigma p^ + P p^ + A't; partial p^'u; the last tile of the
// instance forms alpha.  P p^ of the warp's columns is formed first into
// shared memory (same warp, same columns).
template <class T>
__global__ void __launch_bounds__(GCG_NT, 4) k_gcg_cols(Prob<T, T> P, GcgTiles G, GcgState<T> S, int it,
                                                        int short_p) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ double gcg_dyn[];
  __shared__ double sm[GCG_NT / 32];
  T* sP = reinterpret_cast<T*>(gcg_dyn);   // [max_tile]
  const int tile = blockIdx.x;
  const int inst = G.ct_inst[tile];
  const int par = it & 1;
  if (S.sc_state[par * P.ninst + inst]) return;
  const T beta = (T)S.sc_beta[par * P.ninst + inst];
  const T sig = (T)S.sigma;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t lo = G.ct_lo[tile], hi = G.ct_hi[tile];
  const T2* __restrict__ zp = S.zp;
  const T* __restrict__ t = S.t;
  auto phat = [&](int32_t c) {
    if (c < 0) return T(0);
    const T2 g = __ldg(zp + c);
    return g.x + beta * g.y;
  };
  gcg_p_part(P, G, lo, hi, short_p, phat, sP);
  T pacc = T(0);   // this lane's share of p^'u (lane 0 of each warp)
  gcg_rows_any(
      G.vq_at, P.AT_rp, P.AT_ci, P.AT_v, G.nnz_a, lo + w, hi, GCG_NT / 32, [&](int64_t j) { return S.zp[j]; },
      [&](int32_t c) { return c >= 0 ? __ldg(t + c) : T(0); },
      [&](int64_t j, T2 g, T sum) {
        if (lane == 0) {
          const T pj = g.x + beta * g.y;
          const T uj = sig * pj + sP[j - lo] + sum;
          S.u[j] = uj;
          pacc += pj * uj;
        }
      });
  const T tv[1] = {pacc};
  double acc[1];
  block_sum_t<1>(tv, acc, sm);
  if (threadIdx.x == 0) S.part_a[tile] = acc[0];
  const int tlo = G.it_lo[inst], thi = G.it_hi[inst];
  if (!gcg_last_tile(S.cnt_grp, S.cnt_inst, inst, tile, tlo, thi)) return;
  double* const parts[1] = {S.part_a};
  double pu[1];
  gcg_tile_sum<GCG_NT, 1>(parts, tlo, thi, pu, sm);
  if (threadIdx.x == 0) {
    const double rz = S.sc_rz[par * P.ninst + inst];
    S.sc_alpha[inst] = pu[0] > 0.0 ? rz / pu[0] : 0.0;
  }
}

// update: x += alpha p^, r -= alpha u, z = D^-1 r, p <- p^; the last tile of
// the instance forms r'z, beta and the state of iteration it + 1.
template <class T, int NT = GCG_NT>
__global__ void __launch_bounds__(NT) k_gcg_update(Prob<T, T> P, GcgTiles G, GcgState<T> S, int it) {
  __shared__ double sm[2 * (NT / 32)];
  const int tile = blockIdx.x;
  const int inst = G.ct_inst[tile];
  const int par = it & 1, nxt = (it + 1) & 1;
  const int lo = G.it_lo[inst], hi = G.it_hi[inst];
  const int st = S.sc_state[par * P.ninst + inst];
  if (st) {
    // stopped: carry the scalars into the next parity
    if (tile == lo && threadIdx.x == 0) {
      S.sc_state[nxt * P.ninst + inst] = st;
      S.sc_rz[nxt * P.ninst + inst] = S.sc_rz[par * P.ninst + inst];
      S.sc_beta[nxt * P.ninst + inst] = 0.0;
    }
    return;
  }
  const T beta = (T)S.sc_beta[par * P.ninst + inst];
  const T alpha = (T)S.sc_alpha[inst];
  T a0 = T(0), a1 = T(0);
  for (int64_t j = G.ct_lo[tile] + threadIdx.x; j < G.ct_hi[tile]; j += NT) {
    const auto g = S.zp[j];
    const T pj = g.x + beta * g.y;
    S.x[j] += alpha * pj;
    const T rj = S.r[j] - alpha * S.u[j];
    const T zj = S.dinv[j] * rj;
    typename Vec2<T>::type ng;
    ng.x = zj;
    ng.y = pj;
    S.r[j] = rj;
    S.zp[j] = ng;
    a0 += rj * zj;
    a1 += rj * rj;
  }
  const T tv[2] = {a0, a1};
  double acc[2];
  block_sum_t<2>(tv, acc, sm);
  if (threadIdx.x == 0) {
    S.part_a[tile] = acc[0];
    S.part_b[tile] = acc[1];
  }
  if (!gcg_last_tile(S.cnt_grp, S.cnt_inst, inst, tile, lo, hi)) return;
  double* const parts[2] = {S.part_a, S.part_b};
  double tot[2];
  gcg_tile_sum<NT, 2>(parts, lo, hi, tot, sm);
  if (threadIdx.x == 0) {
    const double rz_old = S.sc_rz[par * P.ninst + inst];
    S.sc_rz[nxt * P.ninst + inst] = tot[0];
    S.sc_beta[nxt * P.ninst + inst] = rz_old != 0.0 ? tot[0] / rz_old : 0.0;
    S.sc_state[nxt * P.ninst + inst] = gcg_next_state(tot[1], S.sc_bb[inst], S.tol, it + 1, S.maxit);
  }
}


// Grid barrier words of the streamed solve (zero before the launch): the
// arrival counter, a spare word, the error word, and the clock cycles a CTA
// may wait at one barrier.
struct GridBar {
  unsigned* arrive;   // zero before the launch
  unsigned* gen;      // zero before the launch
  int32_t* err;       // set to 1 when a wait gave up
  long long limit;    // clock cycles a CTA may wait at one barrier
};

// per-instance CG scalars kept in shared memory by every CTA of the streamed solve
struct GcgScal {
  double gamma, gamma_old, alpha, alpha_old, beta, delta, rr, bb;
  int32_t state;      // 0 iterate, 1 converged, 2 cap reached
  int32_t pad;
};

}  // namespace cosmo
