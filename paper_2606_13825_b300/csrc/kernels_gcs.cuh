// Streamed grid-wide CG for one or a few large instances of the reduced
// system (P + sigma I + A'D(rho)A) x = rhs (Sec. 2.3) at the App. B scale,
// where A and A' are far larger than L2 and every CG iteration streams both
// from HBM once.
//
// Layout (built once per matrix by a plan, Sec. 2.3's operator is fixed
// while rho, sigma and rhs change).  A gathers z over the instance's
// columns, A' gathers t over its rows; a gathered vector that does not fit in
// shared memory next to the streaming buffers is cut into `nseg` equal
// segments.  Each source row is stored once per segment with the entries
// whose index falls in that segment (original order), padded with zero
// values to a multiple of 4 entries ("quads"): a quad never holds two rows.
// qp[h][r] is the first quad of row r's piece in segment h (absolute).
// Quads are stored in chunks of gcs_cq() quads, each chunk one contiguous
// block [values of its quads | column indices of its quads], and the last
// row of every tile is padded to a whole chunk: a tile's piece of a segment
// is a run of whole chunks, and each chunk arrives with one bulk copy of
// 1 KB (float) -- the TMA engine sustains HBM bandwidth with 1 KB requests
// from a few dozen warps, but only about 60% of it with 512-byte ones.
//
// Kernel: one CTA per SM, 24 streaming warps and one control warp.  Each
// streaming warp owns an equal share of its tile's quads per segment and
// streams them through a private ring of chunk buffers filled by
// bulk asynchronous copies (cp.async.bulk, the TMA engine; completion on an
// mbarrier per buffer).  Data in flight lands in shared memory, not in L1,
// so staging the gathered vector in shared memory does not cut the loads in
// flight, and a warp keeps two chunks in flight while it works on a third.
// A lane takes one quad (float) or half a quad (double), gathers from the
// staged vector, and a segmented warp scan over the lanes' row indices sums
// each row piece in a fixed order (bitwise reproducible).  The row a warp's
// share starts inside is summed into a per-warp slot and added after the
// segment in warp order.
//
// Iteration: Jacobi-PCG in the Chronopoulos-Gear arrangement (the iterates
// of textbook PCG in exact arithmetic; s = M p kept by recurrence), with the
// one dot product that needs the matrix-vector product, delta = z'Mz, formed
// from the row phase as sigma ||z||^2 + z'Pz + sum_r rho_r (Az)_r^2:
//
//   R:  t = rho o (A z),  partial sum rho (Az)^2, P z and sigma z'z + z'Pz
//       (z staged per column segment)
//   C:  alpha = gamma / (delta - beta gamma / alpha_old)   (control warp)
//       w = sigma z + P z + A't                  (t staged per row segment)
//       s = w + beta s, p = z + beta p, x += alpha p, r -= alpha s,
//       z = D^-1 r, partial r'z (gamma) and r'r of the CTA's columns
//
// so the update runs in the epilogue of the A' phase and an iteration has two
// grid barriers (after R, after C).  (The pipelined form of Ghysels and
// Vanroose would also give two barriers, but its recurrences for M u and
// M q amplify the rounding of an FP32 matrix-vector product by about 1.3
// per iteration on the App. B systems and break down within tens of
// iterations.)  The control warp sums the partials published before the last
// barrier while the streaming warps stream: gamma, r'r and the stop test in
// R, delta and alpha in C.  Every CTA forms every instance's scalars in the
// same order (identical values and stop decisions, no atomics).  The stop
// test ||r|| <= tol ||rhs|| is taken in R on the residual of the last update,
// so the R phase of the stopping iteration is discarded.  Every wait is
// bounded in clock cycles; a wait that gives up sets the error word, waits
// (bounded) for this CTA's copies in flight and returns.
#pragma once

#include <cooperative_groups.h>

#include "kernels_gcg.cuh"
#include "kernels_tc.cuh"

namespace cosmo {

namespace bulk {

// one bulk copy global -> shared memory of this CTA (TMA engine); `bytes` a
// multiple of 16, both addresses 16-byte aligned; completion counted on mbar
__device__ __forceinline__ void copy(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(tc::smem_u32(dst)), "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar)) : "memory");
}

// arrive on mbar (count 1) and expect `bytes` of transactions in this phase
__device__ __forceinline__ void expect(uint64_t* mbar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}"
               :: "r"(tc::smem_u32(mbar)), "r"(bytes) : "memory");
}

// order this thread's generic-proxy accesses before later async-proxy ones
__device__ __forceinline__ void fence_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// wait for the phase of the given parity; false after `limit` clock cycles.
// Each try may suspend the thread for up to 10 us until the phase completes
// (the warp gives its issue slots to the others instead of spinning).
__device__ __forceinline__ bool wait(uint64_t* mbar, uint32_t parity, long long limit) {
  long long t0 = 0;
  for (int k = 0;; ++k) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(tc::smem_u32(mbar)), "r"(parity), "r"(10000u) : "memory");
    if (done) return true;
    if (k == 0) t0 = clock64();
    else if (clock64() - t0 > limit) return false;
  }
}

}  // namespace bulk

// Phase timer stamps (thread 0 of each CTA, when enabled): 0 iteration start,
// 1 R stage ready, 2 warp 0's R stream done, 3 every warp's R stream done,
// 4 R epilogue done, 5 past the R->C grid barrier, 6 C stage ready, 7 warp
// 0's C stream done, 8 every warp's C stream done, 9 update done (the next
// iteration's 0 is the end of the C->R barrier).
constexpr int GCS_NSTAMP = 10;

constexpr int GCS_WARPS = 24;                    // streaming warps
constexpr int GCS_NT = 32 * GCS_WARPS + 32;      // + the control warp (800 threads, 80 registers each)
constexpr int GCS_MAXSLOT = 6;                   // chunk buffers per streaming warp, at most
// quads per chunk: 128 float or 64 double entries (32 lanes x 16 bytes of values)
template <class T> __host__ __device__ constexpr int gcs_cq() { return sizeof(T) == 4 ? 32 : 16; }
template <class T> __host__ __device__ constexpr int gcs_vbytes() { return gcs_cq<T>() * 4 * (int)sizeof(T); }
template <class T> __host__ __device__ constexpr int gcs_slot() { return gcs_vbytes<T>() + gcs_cq<T>() * 16; }

// segment h of a gathered range [o0, o1) cut into nseg equal parts
__host__ __device__ inline void gcs_seg(int64_t o0, int64_t o1, int nseg, int h, int64_t& lo, int64_t& hi) {
  const int64_t len = o1 - o0, ws = (len + nseg - 1) / nseg;
  lo = o0 + (h * ws < len ? h * ws : len);
  hi = o0 + ((h + 1) * ws < len ? (h + 1) * ws : len);
}

__host__ __device__ inline int64_t gcs_al(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// byte offsets into the kernel's dynamic shared memory; every region starts
// on a 16-byte boundary (the mbarriers and the int64 / double tables need 8,
// the bulk-copy destinations 16)
struct GcsSmem {
  int64_t o_ring, o_mbar, o_stage, o_ps, o_ns, o_sp, o_rho, o_epi, o_headv, o_headr, o_qend_r, o_qend_c, o_qb,
      o_scal, total;
};

// RT: rows of the largest cluster tile, RTo / CTo: of the largest share one
// CTA owns in the epilogues, CTc: rows of A' one CTA streams at most
template <class T>
__host__ __device__ inline GcsSmem gcs_smem(int nslot, int64_t stage_len, int64_t RT, int64_t CTc, int64_t RTo,
                                            int64_t CTo, int ninst) {
  GcsSmem s{};
  int64_t o = 0;
  s.o_ring = o;   o += (int64_t)GCS_WARPS * nslot * gcs_slot<T>();
  s.o_mbar = o;   o = gcs_al(o + 8 * (GCS_WARPS * nslot + 1), 128);
  s.o_stage = o;  o += gcs_al(stage_len * (int64_t)sizeof(T), 16);
  s.o_ps = o;     o += gcs_al(RT * (int64_t)sizeof(T), 16);
  s.o_ns = o;     o += gcs_al(CTc * (int64_t)sizeof(T), 16);
  s.o_sp = o;     o += gcs_al(CTo * (int64_t)sizeof(T), 16);
  s.o_rho = o;    o += gcs_al(RTo * (int64_t)sizeof(T), 16);
  s.o_epi = o;    o += gcs_al(6 * CTo * (int64_t)sizeof(T), 16);
  s.o_headv = o;  o += gcs_al(GCS_WARPS * (int64_t)sizeof(T), 16);
  s.o_headr = o;  o += gcs_al(GCS_WARPS * 4, 16);
  s.o_qend_r = o; o += gcs_al(RT * 4, 16);
  s.o_qend_c = o; o += gcs_al(CTc * 4, 16);
  s.o_qb = o;     o += 16;
  s.o_scal = o;   o += (int64_t)ninst * (int64_t)sizeof(GcgScal);
  s.total = gcs_al(o, 16);
  return s;
}

template <class T>
struct GcsLayout {
  const unsigned char* data;  // [quads / gcs_cq] chunks of gcs_chunk_bytes; padding
                              // entries: value 0, the segment's first index
  const int64_t* qp;          // [nseg][rows + 1] absolute first quad of each row piece
  int32_t nseg;
  int64_t rows;
};

template <class T> __host__ __device__ constexpr int gcs_chunk_bytes() { return gcs_slot<T>(); }

// byte offsets of entry e's value and column index in a layout
template <class T> __host__ __device__ inline int64_t gcs_val_at(int64_t e) {
  const int64_t q = e >> 2;
  return (q / gcs_cq<T>()) * gcs_chunk_bytes<T>() + (q % gcs_cq<T>()) * 4 * (int64_t)sizeof(T) + (e & 3) * (int64_t)sizeof(T);
}
template <class T> __host__ __device__ inline int64_t gcs_col_at(int64_t e) {
  const int64_t q = e >> 2;
  return (q / gcs_cq<T>()) * gcs_chunk_bytes<T>() + gcs_vbytes<T>() + (q % gcs_cq<T>()) * 16 + (e & 3) * 4;
}

// Tiles are per cluster (index blockIdx.x / CS; G's row / column tile
// arrays).  R: CTA rank h of a cluster streams segment h of the rows of its
// tile (A's layout has nseg == CS; the row sums are combined over the
// cluster).  C, when the instance's whole t fits shared memory (c_split 0):
// every CTA stages all of t and rank h streams the rows of A' of the h-th
// share of the tile's columns (A''s layout has one segment, tiles = the
// CTAs' shares), so no combination is needed; otherwise (c_split 1) like R,
// segment h of t and of the rows of A' of the whole tile, combined over the
// cluster.  Rank h owns the h-th share of the tile's rows and columns in the
// epilogues.
template <class T>
struct GcsArgs {
  GcsLayout<T> LR;       // rows of A by column segment (R phase)
  GcsLayout<T> LC;       // rows of A' by row segment (C phase)
  const T* rhs; T* x; const T* rho; const T* dinv; double sigma;
  T *r, *z, *p, *s, *t;  // z and t padded to whole 16-byte groups
  double* part_r;        // [grid] sum rho (Az)^2 of the CTA's rows
  double* part_d;        // [grid] sigma z'z + z'Pz of the CTA's columns
  double* part_c;        // [2][2][grid] r'z, r'r of the CTA's columns (by iteration parity)
  const int32_t* cr_lo;  // [ninst] first CTA owning rows of the instance
  const int32_t* cr_hi;  // [ninst] one past the last
  const int32_t* cc_lo;  // [ninst] first CTA owning columns of the instance
  const int32_t* cc_hi;
  int32_t* iters;        // [ninst] or null
  unsigned long long* ts;  // phase timer: [ts_iters][GCS_NSTAMP][grid] globaltimer stamps, or null
  int32_t ts_iters;
  double tol;
  int32_t maxit;
  int32_t short_p;       // P rows of at most 16 entries
  int32_t p_diag;        // P diagonal (or absent): P z of the owned columns is
                         // formed where z is, in the update
  const T* pd;           // [n] P_jj when p_diag
  int32_t nslot;         // chunk buffers per streaming warp
  int32_t c_split;       // C by segment of t (1) or over the whole t (0)
  int32_t RT, CT;        // largest cluster tile: rows / columns
  int32_t RTo, CTo;      // largest owned share
  GcsSmem sm;
  long long wait_limit;  // clock cycles one wait may take
};

// ---- plan-time layout construction ----------------------------------------

// cnt[h * rows + r] = entries of row r whose index lies in segment h of the
// row's instance (indices outside the instance are dropped); one warp per row
__global__ void k_gcs_count(int64_t rows, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            int32_t ninst, const int64_t* __restrict__ row_inst_off,
                            const int64_t* __restrict__ gath_off, int32_t nseg, int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  int lo = 0, hi = ninst;   // instance of row r
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (row_inst_off[mid] <= r) lo = mid; else hi = mid;
  }
  const int64_t o0 = gath_off[lo], o1 = gath_off[lo + 1];
  const int64_t e0 = rp[r], e1 = rp[r + 1];
  for (int h = 0; h < nseg; ++h) {
    int64_t s0, s1;
    gcs_seg(o0, o1, nseg, h, s0, s1);
    int c = 0;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      const int64_t k = ci[e];
      c += (k >= s0 && k < s1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[(int64_t)h * rows + r] = c;
  }
}

// stable compaction of each row's entries into its piece of every segment,
// then zero padding to the piece's end; one warp per row
template <class T>
__global__ void k_gcs_scatter(int64_t rows, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const T* __restrict__ v, int32_t ninst, const int64_t* __restrict__ row_inst_off,
                              const int64_t* __restrict__ gath_off, int32_t nseg, const int64_t* __restrict__ qp,
                              unsigned char* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  int lo = 0, hi = ninst;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (row_inst_off[mid] <= r) lo = mid; else hi = mid;
  }
  const int64_t o0 = gath_off[lo], o1 = gath_off[lo + 1];
  const int64_t e0 = rp[r], e1 = rp[r + 1];
  for (int h = 0; h < nseg; ++h) {
    int64_t s0, s1;
    gcs_seg(o0, o1, nseg, h, s0, s1);
    const int64_t* q = qp + (int64_t)h * (rows + 1);
    int64_t pos = 4 * q[r];
    const int64_t end = 4 * q[r + 1];
    for (int64_t eb = e0; eb < e1; eb += 32) {
      const int64_t e = eb + lane;
      int32_t k = 0;
      bool in = false;
      if (e < e1) {
        k = ci[e];
        in = k >= s0 && k < s1;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int64_t at = pos + __popc(mask & ((1u << lane) - 1u));
        *reinterpret_cast<T*>(out + gcs_val_at<T>(at)) = v[e];
        *reinterpret_cast<int32_t*>(out + gcs_col_at<T>(at)) = k;
      }
      pos += __popc(mask);
    }
    for (int64_t at = pos + lane; at < end; at += 32) {
      *reinterpret_cast<T*>(out + gcs_val_at<T>(at)) = T(0);
      *reinterpret_cast<int32_t*>(out + gcs_col_at<T>(at)) = (int32_t)s0;
    }
  }
}

// d_j = P_jj + sigma + sum_e v_e^2 rho_{c_e} over row j of A' (the layout's
// pieces; padding contributes zero); one warp per column
template <class T>
__global__ void k_gcs_precond(int64_t n, GcsLayout<T> LC, const int64_t* __restrict__ P_rp,
                              const int32_t* __restrict__ P_ci, const T* __restrict__ P_v, double sigma,
                              const T* __restrict__ rho, T* __restrict__ dinv) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  T acc = T(0);
  for (int h = 0; h < LC.nseg; ++h) {
    const int64_t* q = LC.qp + (int64_t)h * (n + 1);
    for (int64_t e = 4 * q[j] + lane; e < 4 * q[j + 1]; e += 32) {
      const T a = *reinterpret_cast<const T*>(LC.data + gcs_val_at<T>(e));
      acc += a * a * rho[*reinterpret_cast<const int32_t*>(LC.data + gcs_col_at<T>(e))];
    }
  }
  T pd = T(0);
  if (P_rp) {
    for (int64_t e = P_rp[j] + lane; e < P_rp[j + 1]; e += 32)
      if (P_ci[e] == j) pd += P_v[e];
  }
  acc += pd;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const T d = acc + (T)sigma;
    dinv[j] = d > T(0) ? T(1) / d : T(0);
  }
}

// ---- the solve --------------------------------------------------------------

template <class T, int CS>
__global__ void __launch_bounds__(GCS_NT, 1) k_gcg_stream(Prob<T, T> P, GcgTiles G, GcsArgs<T> S, GridBar B) {
  extern __shared__ __align__(128) unsigned char gcs_dyn[];
  constexpr int CQ = gcs_cq<T>();
  constexpr int VB = gcs_vbytes<T>();
  constexpr int SLOT = gcs_slot<T>();
  constexpr int E = 16 / (int)sizeof(T);          // elements per 16-byte group
  constexpr int UPQ = sizeof(T) == 4 ? 1 : 2;     // lanes per quad
  // shared-memory arrays, addressed from the offsets each time they are
  // used (kernel parameters: no registers held across the loops)
#define GCS_AT(type, field) reinterpret_cast<type*>(gcs_dyn + S.sm.field)
#define ring GCS_AT(unsigned char, o_ring)
#define mbar GCS_AT(uint64_t, o_mbar)
#define mstage (GCS_AT(uint64_t, o_mbar) + GCS_WARPS * S.nslot)
#define stage GCS_AT(T, o_stage)
#define ps GCS_AT(T, o_ps)
#define ns GCS_AT(T, o_ns)
#define sP GCS_AT(T, o_sp)
#define rho_s GCS_AT(T, o_rho)
#define epi GCS_AT(T, o_epi)
#define headv GCS_AT(T, o_headv)
#define headr GCS_AT(int32_t, o_headr)
#define qend_r GCS_AT(int32_t, o_qend_r)
#define qend_c GCS_AT(int32_t, o_qend_c)
#define qb GCS_AT(int64_t, o_qb)
#define sc GCS_AT(GcgScal, o_scal)
  __shared__ double red[2][GCS_WARPS + 1];
  __shared__ int s_done, s_ok;
  __shared__ int s_bad[2];   // a wait of this CTA gave up, by decision-point parity

  // the CTA's tile constants live in shared memory and are read where used,
  // so that the streaming loop does not hold them in registers
  __shared__ int64_t s_t64[11];
  __shared__ int s_t32[9];
#define clo s_t64[0]
#define chi s_t64[1]
#define rlo s_t64[2]
#define rhi s_t64[3]
#define r_c0 s_t64[4]
#define r_c1 s_t64[5]
#define c_r0 s_t64[6]
#define c_r1 s_t64[7]
#define oc0 s_t64[8]
#define oc1 s_t64[9]
#define nr s_t32[0]
#define nc s_t32[1]
#define orl s_t32[2]
#define nor s_t32[3]
#define ocl s_t32[4]
#define noc s_t32[5]
#define cinst s_t32[6]
#define rinst s_t32[7]
#define ncs s_t32[8]    // rows of A' this CTA streams in C
#define cb0 s_t64[10]   // the first of them
  const int b = blockIdx.x, ninst = P.ninst, NS = S.nslot;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const bool streamer = wp < GCS_WARPS;
  int rank = 0;
  if constexpr (CS > 1) rank = (int)cooperative_groups::this_cluster().block_rank();
  const bool has_r = b / CS < G.nrt, has_c = b / CS < G.nct;
  if (threadIdx.x == 0) {
    const int cl = b / CS;
    cinst = has_c ? G.ct_inst[cl] : 0;
    rinst = has_r ? G.rt_inst[cl] : 0;
    clo = has_c ? G.ct_lo[cl] : 0;
    chi = has_c ? G.ct_hi[cl] : 0;
    rlo = has_r ? G.rt_lo[cl] : 0;
    rhi = has_r ? G.rt_hi[cl] : 0;
    nr = (int)(rhi - rlo);
    nc = (int)(chi - clo);
    // this CTA's shares of the tile's rows / columns in the epilogues
    orl = nr * rank / CS;
    nor = nr * (rank + 1) / CS - orl;
    ocl = nc * rank / CS;
    noc = nc * (rank + 1) / CS - ocl;
    oc0 = clo + ocl;
    oc1 = oc0 + noc;
    // this CTA's segment of z (R) and of t (C)
    int64_t a0 = 0, a1 = 0;
    if (has_r) gcs_seg(P.col_off[rinst], P.col_off[rinst + 1], CS, rank, a0, a1);
    r_c0 = a0; r_c1 = a1;
    if (S.c_split) {
      a0 = a1 = 0;
      if (has_c) gcs_seg(P.row_off[cinst], P.row_off[cinst + 1], CS, rank, a0, a1);
      c_r0 = a0; c_r1 = a1;
      ncs = nc;
      cb0 = clo;
    } else {
      c_r0 = has_c ? P.row_off[cinst] : 0;   // the instance's whole t
      c_r1 = has_c ? P.row_off[cinst + 1] : 0;
      ncs = noc;
      cb0 = oc0;
    }
  }
  __syncthreads();
  const int64_t m_tot = P.m_total, n_tot = P.n_total;

  // ---- per-CTA tables (fixed for the whole solve): segment `rank` ----
  {
    const int64_t* q = S.LR.qp + (int64_t)rank * (m_tot + 1);
    const int64_t base = has_r ? q[rlo] : 0;
    if (threadIdx.x == 0) qb[0] = base;
    for (int k = threadIdx.x; k < nr; k += GCS_NT) qend_r[k] = (int32_t)(q[rlo + k + 1] - base);
  }
  {
    // segment `rank` of the tile's columns, or the one segment of the CTA's own
    const int64_t* q = S.LC.qp + (S.c_split ? (int64_t)rank * (n_tot + 1) : 0);
    const int64_t base = has_c ? q[cb0] : 0;
    if (threadIdx.x == 0) qb[1] = base;
    for (int k = threadIdx.x; k < ncs; k += GCS_NT) qend_c[k] = (int32_t)(q[cb0 + k + 1] - base);
  }
  for (int k = threadIdx.x; k < nor; k += GCS_NT) rho_s[k] = S.rho[rlo + orl + k];
  for (int k = threadIdx.x; k < nr; k += GCS_NT) ps[k] = T(0);
  for (int k = threadIdx.x; k < ncs; k += GCS_NT) ns[k] = T(0);
  for (int i = threadIdx.x; i < ninst; i += GCS_NT) {
    sc[i].state = 0;
    sc[i].alpha = sc[i].alpha_old = sc[i].beta = sc[i].gamma = sc[i].gamma_old = 0.0;
    sc[i].delta = sc[i].rr = sc[i].bb = 0.0;
  }
  if (streamer && lane == 0)
    for (int k = 0; k < NS; ++k) tc::mbar_init(mbar + wp * NS + k, 1);
  if (threadIdx.x == 0) {
    tc::mbar_init(mstage, 1);
    s_done = 0;
    s_ok = 1;
    s_bad[0] = s_bad[1] = 0;
  }
  bulk::fence_init();
  // every CTA of the cluster is running (and initialised) before any
  // distributed shared-memory access
  auto csync = [&]() {
    if constexpr (CS > 1) cooperative_groups::this_cluster().sync();
    else __syncthreads();
  };
  csync();

  // segment 0 = R (A's rows of the tile), 1 = C (A''s rows = the tile's columns)
  // (a tile's quads, and so its chunks, fit 31 bits: qend is int32)
  auto seg_total = [&](int sidx) -> int32_t {
    if (sidx == 0) return nr > 0 ? qend_r[nr - 1] : 0;
    return ncs > 0 ? qend_c[ncs - 1] : 0;
  };
  auto warp_chunks = [&](int sidx, int32_t& c0, int32_t& c1) {
    const int64_t nch = (seg_total(sidx) + CQ - 1) / CQ;
    c0 = (int32_t)(nch * wp / GCS_WARPS);
    c1 = (int32_t)(nch * (wp + 1) / GCS_WARPS);
  };

  // ---- producer: this warp's chunks of R then C, cyclically ----
  int p_sidx = 1;
  int32_t p_c = 0, p_c1 = 0;
  bool any_chunks = false;
  if (streamer) {
    for (int sidx = 0; sidx < 2; ++sidx) {
      int32_t c0, c1;
      warp_chunks(sidx, c0, c1);
      any_chunks |= c1 > c0;
    }
  }
  auto advance = [&]() {
    ++p_c;
    while (p_c >= p_c1) {
      p_sidx ^= 1;
      warp_chunks(p_sidx, p_c, p_c1);
    }
  };
#define wring (ring + wp * NS * SLOT)   // this warp's buffers
#define wmbar (mbar + wp * NS)
  // lane 0 issues the producer's current chunk (always whole; the tile's
  // piece starts on a chunk) into `slot` with one bulk copy, then advances
  auto issue = [&](int slot) {
    if (lane == 0) {
      const unsigned char* src = (p_sidx == 0 ? S.LR.data : S.LC.data) + (qb[p_sidx] / CQ + p_c) * SLOT;
      bulk::fence_shared();
      bulk::expect(wmbar + slot, SLOT);
      bulk::copy(wring + slot * SLOT, src, SLOT, wmbar + slot);
    }
    advance();
  };
  int rslot = 0;          // next buffer to consume and the parity of its phase
  uint32_t rphase = 0;
  if (streamer && any_chunks) {
    advance();
    for (int k = 0; k < NS; ++k) issue(k);
  }
  uint32_t stage_uses = 0;
  bool bad = false;       // a wait of this thread gave up
  int dp = 0;             // decision points passed (parity selects s_bad)

  auto fail = [&]() {
    bad = true;
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> e(*B.err);
    e.store(1, cuda::memory_order_relaxed);
    s_bad[dp & 1] = 1;
  };
  // at a decision point, after csync(): did any CTA of the cluster fail in
  // the phase that just ended?  (partners write the other parity slot in the
  // next phase, so every CTA reads the same values)
  auto cluster_bad = [&]() -> bool {
    int any = s_bad[dp & 1];
    if constexpr (CS > 1) {
      cooperative_groups::cluster_group g = cooperative_groups::this_cluster();
      for (int q = 0; q < CS; ++q) any |= *g.map_shared_rank(&s_bad[dp & 1], q);
    }
    ++dp;
    return any != 0;
  };
  // leave: one more cluster barrier (partners may still read this CTA's
  // shared memory until they reach it), then wait for the copies in flight
  auto leave = [&]() {
    csync();
    if (streamer && any_chunks) {
      for (int k = 0; k < NS; ++k) {
        const int sl = rslot + k;
        bulk::wait(wmbar + (sl >= NS ? sl - NS : sl), rphase ^ (sl >= NS ? 1u : 0u), S.wait_limit);
      }
    }
    if (bad && threadIdx.x == 0 && stage_uses > 0) bulk::wait(mstage, (stage_uses - 1) & 1, S.wait_limit);
  };

  // grid barrier: thread 0 of every CTA adds to the global counter (a
  // fire-and-forget release add) and polls it (acquire) until every CTA has
  // arrived; the CTA barrier then extends that to its other threads.  A CTA
  // passes only when all CTAs have finished the phase, including their
  // reads of partner CTAs' shared memory.  Gives up after the wait limit or
  // when the error word is set; the caller then marks the CTA bad and the
  // cluster leaves together at its next decision point.
  unsigned epoch = 0;
  auto grid_sync = [&]() -> bool {
    __syncthreads();
    if (threadIdx.x == 0) {
      ++epoch;
      const unsigned target = epoch * gridDim.x;
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(B.arrive) : "memory");
      int ok = 1;
      long long t0 = 0;
      for (int k = 0;; ++k) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(B.arrive) : "memory");
        if (v >= target) break;
        if (k == 0) t0 = clock64();
        if ((k & 63) == 63) {
          int e;
          asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(e) : "l"(B.err) : "memory");
          if (e != 0 || clock64() - t0 > B.limit) {
            ok = 0;
            break;
          }
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  };

  // stage gathered[lo, hi) (16-byte groups) into shared memory: thread 0
  // issues the copy, the streaming threads wait in stage_wait.  Returns the
  // group-aligned base index.
  auto stage_issue = [&](const T* src, int64_t lo, int64_t hi) -> int32_t {
    const int64_t gb = lo & ~(int64_t)(E - 1);
    const int64_t bytes = gcs_al(hi - gb, E) * (int64_t)sizeof(T);
    if (hi > lo && threadIdx.x == 0) {
      bulk::fence_global();
      bulk::fence_shared();
      bulk::expect(mstage, (uint32_t)bytes);
      for (int64_t o = 0; o < bytes; o += 32768)
        bulk::copy(reinterpret_cast<unsigned char*>(stage) + o, reinterpret_cast<const unsigned char*>(src + gb) + o,
                   (uint32_t)min((int64_t)32768, bytes - o), mstage);
    }
    return (int32_t)gb;
  };
  auto stage_wait = [&](int64_t lo, int64_t hi) {
    if (hi <= lo) return;
    if (streamer && !bad && !bulk::wait(mstage, stage_uses & 1, S.wait_limit)) fail();
    ++stage_uses;
  };

  // consume this warp's chunks of segment sidx: acc[k] += row piece sums of
  // the tile's rows (relative index k), gathered from stage (base gb).
  // Lanes keep running sums of the current row (acc0) and the next (acc1);
  // a row's lanes are summed (fixed butterfly) when the row ends.  A chunk
  // spanning three or more rows takes a segmented scan instead.  The order
  // of every sum is fixed by the layout: results are bitwise reproducible.
  auto consume = [&](int sidx, const int32_t* qend, int nrow, T* acc, int32_t gb) {
    int32_t c0, c1;
    warp_chunks(sidx, c0, c1);
    if (lane == 0) headr[wp] = -1;
    if (c0 >= c1) return;
    // the row holding the warp's first quad, and whether it began earlier
    const int32_t qw = c0 * CQ;
    int lo = 0, hi = nrow - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (qend[mid] > qw) hi = mid; else lo = mid + 1;
    }
    const int hrow = lo;
    const bool hstart = (hrow > 0 ? qend[hrow - 1] : 0) < qw;
    if (lane == 0) {
      headv[wp] = T(0);
      headr[wp] = hstart ? hrow : -1;
    }
    __syncwarp();
    const T* st = stage - gb;
    const int32_t qt = seg_total(sidx);
    const int quad = lane / UPQ;
    int rrow = hrow;
    T acc0 = T(0), acc1 = T(0);
    auto target = [&](int row) { return (hstart && row == hrow) ? headv + wp : acc + row; };
    for (int32_t c = c0; c < c1; ++c) {
      if (!bad && !bulk::wait(wmbar + rslot, rphase, S.wait_limit)) fail();
      if (bad) return;
      // the lane's entries into registers, then the buffer is refilled at
      // once: the warp keeps every buffer in flight while it computes
      const unsigned char* buf = wring + rslot * SLOT;
      const int32_t cq = c * CQ;
      const int nq = min(CQ, qt - cq);
      const bool valid = quad < nq;
      using VV = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
      using VI = typename std::conditional<sizeof(T) == 4, int4, int2>::type;
      const VV v = reinterpret_cast<const VV*>(buf)[lane];
      const VI ci = reinterpret_cast<const VI*>(buf + VB)[lane];
      if constexpr (sizeof(T) == 4)
        asm volatile("" :: "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(ci.x), "r"(ci.y), "r"(ci.z), "r"(ci.w));
      else
        asm volatile("" :: "d"(v.x), "d"(v.y), "r"(ci.x), "r"(ci.y));
      __syncwarp();
      const int used = rslot;
      if (++rslot == NS) { rslot = 0; rphase ^= 1u; }
      issue(used);
      T d = T(0);
      int k = 0x7fffffff;
      if (valid) {
        if constexpr (sizeof(T) == 4) d = v.x * st[ci.x] + v.y * st[ci.y] + v.z * st[ci.z] + v.w * st[ci.w];
        else d = v.x * st[ci.x] + v.y * st[ci.y];
        k = rrow;
        while (k < nrow - 1 && qend[k] <= cq + quad) ++k;
      }
      const int kl = __shfl_sync(0xffffffffu, k, nq * UPQ - 1);   // row of the chunk's last quad
      if (kl <= rrow + 1) {
        if (k == rrow) acc0 += d; else acc1 += d;   // (invalid lanes add d = 0)
        if (kl > rrow) {                             // row rrow ended inside the chunk
          const T sum = warp_allsum(acc0);
          if (lane == 0) *target(rrow) += sum;
          acc0 = acc1;
          acc1 = T(0);
          rrow = kl;
        }
        if (qend[rrow] == cq + nq) {                 // row rrow ends with the chunk
          const T sum = warp_allsum(acc0);
          if (lane == 0) *target(rrow) += sum;
          acc0 = T(0);
          if (rrow < nrow - 1) ++rrow;
        }
      } else {
        // three or more rows: the running sum first, then a segmented
        // inclusive scan over the lanes keyed by row
        const T sum = warp_allsum(acc0);
        if (lane == 0) *target(rrow) += sum;
        acc0 = T(0);
        __syncwarp();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const T up = __shfl_up_sync(0xffffffffu, d, o);
          const int ku = __shfl_up_sync(0xffffffffu, k, o);
          if (lane >= o && ku == k) d += up;
        }
        const int knext = __shfl_down_sync(0xffffffffu, k, 1);
        if (valid && (lane == 31 || knext != k)) *target(k) += d;
        __syncwarp();
        rrow = kl;
      }
    }
    // the running sum of the last row (it continues in the next warp's share)
    const T sum = warp_allsum(acc0);
    if (lane == 0 && sum != T(0)) *target(rrow) += sum;
    __syncwarp();
  };

  // add the warps' head slots in warp order (one thread), after the segment
  auto fixup = [&](T* acc) {
    if (threadIdx.x == 0)
      for (int w2 = 0; w2 < GCS_WARPS; ++w2)
        if (headr[w2] >= 0) acc[headr[w2]] += headv[w2];
  };

  // sum over the cluster's CTAs (rank order) of their partial array `a` at k
  auto cluster_total = [&](T* a, int k) -> T {
    if constexpr (CS == 1) {
      return a[k];
    } else {
      cooperative_groups::cluster_group g = cooperative_groups::this_cluster();
      T v = T(0);
#pragma unroll
      for (int q = 0; q < CS; ++q) v += g.map_shared_rank(a, q)[k];
      return v;
    }
  };

  // R (control warp): gamma and r'r of the last update, the stop test, beta
  auto control_r = [&](int it) {
    const double* pc = S.part_c + (int64_t)(it & 1) * 2 * gridDim.x;
    int running = 0;
    for (int i = 0; i < ninst; ++i) {
      if (sc[i].state != 0) continue;
      double g = 0.0, rr = 0.0;
      for (int k = S.cc_lo[i] + lane; k < S.cc_hi[i]; k += 32) {
        g += __ldcg(pc + k);
        rr += __ldcg(pc + gridDim.x + k);
      }
      g = warp_sum(g);
      rr = warp_sum(rr);
      if (lane == 0) {
        GcgScal& c = sc[i];
        if (it == 0) c.bb = rr;
        int stt = 0;
        if (rr <= S.tol * S.tol * c.bb || !(rr == rr)) stt = 1;
        else if (it >= S.maxit) stt = 2;
        if (stt) {
          c.state = stt;
          if (b == 0 && S.iters) S.iters[i] = it;
        } else {
          c.beta = it > 0 && c.gamma_old != 0.0 ? g / c.gamma_old : 0.0;
          c.gamma = g;
          c.rr = rr;
        }
      }
      __syncwarp();
      running += sc[i].state == 0;
    }
    if (lane == 0) s_done = running == 0;
  };
  // C (control warp): delta = z'Mz from the R partials, alpha
  auto control_c = [&](int it) {
    for (int i = 0; i < ninst; ++i) {
      if (sc[i].state != 0) continue;
      double dl = 0.0;
      for (int k = S.cr_lo[i] + lane; k < S.cr_hi[i]; k += 32) dl += __ldcg(S.part_r + k);
      for (int k = S.cc_lo[i] + lane; k < S.cc_hi[i]; k += 32) dl += __ldcg(S.part_d + k);
      dl = warp_sum(dl);
      if (lane == 0) {
        GcgScal& c = sc[i];
        const double den = dl - (it > 0 && c.alpha_old != 0.0 ? c.beta * c.gamma / c.alpha_old : 0.0);
        c.delta = dl;
        c.alpha = den > 0.0 ? c.gamma / den : 0.0;
        c.alpha_old = c.alpha;
        c.gamma_old = c.gamma;
      }
      __syncwarp();
    }
  };

  // CTA sum of two per-thread values in a fixed order (warp sums in T, the
  // warps' values combined in double by warp 0); warp 0 gets the totals
  auto cta_sum2 = [&](T v0, T v1, double& t0, double& t1) {
    v0 = warp_allsum(v0);
    v1 = warp_allsum(v1);
    if (lane == 0) { red[0][wp] = (double)v0; red[1][wp] = (double)v1; }
    __syncthreads();
    if (wp == 0) {
      t0 = warp_sum(lane <= GCS_WARPS ? red[0][lane] : 0.0);
      t1 = warp_sum(lane <= GCS_WARPS ? red[1][lane] : 0.0);
    }
  };


  // ---- zero start (owned columns): x = 0, r = rhs, z = D^-1 rhs, p = s = 0 ----
  {
    T a0 = T(0), a1 = T(0);
    for (int64_t j = oc0 + threadIdx.x; j < oc1; j += GCS_NT) {
      const T bj = S.rhs[j], zj = S.dinv[j] * bj;
      S.x[j] = T(0); S.r[j] = bj; S.z[j] = zj; S.p[j] = T(0); S.s[j] = T(0);
      if (S.p_diag) sP[j - oc0] = S.pd[j] * zj;
      a0 += bj * zj;
      a1 += bj * bj;
    }
    double t0 = 0.0, t1 = 0.0;
    cta_sum2(a0, a1, t0, t1);
    if (threadIdx.x == 0) { S.part_c[b] = t0; S.part_c[gridDim.x + b] = t1; }
  }
  if (!grid_sync()) fail();

  auto stamp = [&](int it, int k) {
    if (S.ts && threadIdx.x == 0 && it < S.ts_iters) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      S.ts[((int64_t)it * GCS_NSTAMP + k) * gridDim.x + b] = t;
    }
  };

  for (int it = 0;; ++it) {
    stamp(it, 0);
    // ---- R: partial (A z) of the cluster's rows over this CTA's segment ----
    // (the stage copy runs while P z is formed; the partner CTAs finished
    // reading ps and ns before the last grid barrier)
    const int32_t gbr = has_r ? stage_issue(S.z, r_c0, r_c1) : 0;
    for (int k = threadIdx.x; k < nr; k += GCS_NT) ps[k] = T(0);
    for (int k = threadIdx.x; k < ncs; k += GCS_NT) ns[k] = T(0);
    if (!S.p_diag)
      gcg_p_part(P, G, oc0, oc1, S.short_p, [&](int32_t c) { return c >= 0 ? __ldcg(S.z + c) : T(0); }, sP);
    else
      __syncthreads();   // the resets above precede the accumulation
    if (has_r) stage_wait(r_c0, r_c1);
    stamp(it, 1);
    if (streamer) {
      if (has_r && !bad) consume(0, qend_r, nr, ps, gbr);
      stamp(it, 2);
    } else {
      control_r(it);
      // the epilogues' operands of the owned columns: z, s, p, x, r, D^-1
      // (unchanged until the update at the end of C)
      const int CTo = S.CTo;
      for (int k = lane; k < noc; k += 32) {
        const int64_t j = oc0 + k;
        const T zj = S.z[j], sj = S.s[j], pj = S.p[j], xj = S.x[j], rj = S.r[j], dj = S.dinv[j];
        epi[k] = zj; epi[CTo + k] = sj; epi[2 * CTo + k] = pj;
        epi[3 * CTo + k] = xj; epi[4 * CTo + k] = rj; epi[5 * CTo + k] = dj;
      }
    }
    __syncthreads();
    if (has_r) fixup(ps);
    csync();   // every CTA's partial row sums are complete
    stamp(it, 3);
    if (cluster_bad() || s_done) { leave(); return; }
    {
      // owned rows: t = rho o (A z); partials sum rho (Az)^2 (rows),
      // sigma z'z + z'Pz (owned columns)
      T a0 = T(0), a1 = T(0);
      for (int k = threadIdx.x; k < nor; k += GCS_NT) {
        const T az = cluster_total(ps, orl + k), tk = rho_s[k] * az;
        S.t[rlo + orl + k] = tk;
        a0 += tk * az;
      }
      const T sig = (T)S.sigma;
      for (int k = threadIdx.x; k < noc; k += GCS_NT) {
        const T zj = epi[k];
        a1 += zj * (sig * zj + sP[k]);
      }
      double t0 = 0.0, t1 = 0.0;
      cta_sum2(a0, a1, t0, t1);
      if (threadIdx.x == 0) { S.part_r[b] = t0; S.part_d[b] = t1; }
    }
    stamp(it, 4);
    if (!grid_sync()) fail();
    stamp(it, 5);

    // ---- C: (A't) of the CTA's own columns over the whole t, or the partial
    // of the tile's columns over this CTA's segment of t ----
    const int32_t gbc = has_c ? stage_issue(S.t, c_r0, c_r1) : 0;
    if (has_c) stage_wait(c_r0, c_r1);
    stamp(it, 6);
    if (streamer) {
      if (has_c && !bad) consume(1, qend_c, ncs, ns, gbc);
      stamp(it, 7);
    } else {
      control_c(it);
    }
    __syncthreads();
    if (has_c) fixup(ns);
    csync();   // every CTA's partial column sums are complete (split C)
    stamp(it, 8);
    if (cluster_bad()) { leave(); return; }

    // ---- update of the owned columns; partials r'z, r'r ----
    {
      T a0 = T(0), a1 = T(0);
      const bool upd = has_c && sc[cinst].state == 0;
      if (upd) {
        const T alpha = (T)sc[cinst].alpha, beta = (T)sc[cinst].beta, sig = (T)S.sigma;
        const int CTo = S.CTo;
        for (int k = threadIdx.x; k < noc; k += GCS_NT) {
          const int64_t j = oc0 + k;
          const T zj = epi[k];
          const T wj = sig * zj + sP[k] + (S.c_split ? cluster_total(ns, ocl + k) : ns[k]);
          const T sj = wj + beta * epi[CTo + k];
          const T pj = zj + beta * epi[2 * CTo + k];
          S.s[j] = sj;
          S.p[j] = pj;
          S.x[j] = epi[3 * CTo + k] + alpha * pj;
          const T rj = epi[4 * CTo + k] - alpha * sj;
          const T zn = epi[5 * CTo + k] * rj;
          S.r[j] = rj;
          S.z[j] = zn;
          if (S.p_diag) sP[k] = S.pd[j] * zn;   // P z of the next iteration
          a0 += rj * zn;
          a1 += rj * rj;
        }
      }
      double t0 = 0.0, t1 = 0.0;
      cta_sum2(a0, a1, t0, t1);
      if (threadIdx.x == 0 && upd) {
        double* pc = S.part_c + (int64_t)((it + 1) & 1) * 2 * gridDim.x;
        pc[b] = t0;
        pc[gridDim.x + b] = t1;
      }
    }
    stamp(it, 9);
    if (!grid_sync()) fail();
  }
#undef wmbar
#undef wring
#undef cb0
#undef ncs
#undef rinst
#undef cinst
#undef noc
#undef ocl
#undef nor
#undef orl
#undef nc
#undef nr
#undef oc1
#undef oc0
#undef c_r1
#undef c_r0
#undef r_c1
#undef r_c0
#undef rhi
#undef rlo
#undef chi
#undef clo
#undef sc
#undef qb
#undef qend_c
#undef qend_r
#undef headr
#undef headv
#undef epi
#undef rho_s
#undef sP
#undef ns
#undef ps
#undef stage
#undef mstage
#undef mbar
#undef ring
#undef GCS_AT
}

}  // namespace cosmo
