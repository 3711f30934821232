// Host runtime of the C ABI declared in include/cosmo_du.h: problem
// validation, batch construction (A' in CSR, cone schedules, row/column
// instance maps), the tape of the unrolled iteration (with checkpoint
// segments), the forward/backward launch sequences, and CUDA-graph capture.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/cosmo_du.h"
#include "common.cuh"
#include "kernels_psd.cuh"
#include "kernels_jt2.cuh"
#include "kernels_tql.cuh"
#include "kernels_gcg.cuh"
#include "kernels_gcs.cuh"
#include "kernels_tc.cuh"
#include "kernels_vec.cuh"
#include "kernels_ws.cuh"
#include "kernels_pol.cuh"
#include "kernels_ws_tc.cuh"
#include "kernels_persist.cuh"
#include "kernels_tpb.cuh"

using namespace cosmo;

// ------------------------------------------------------------ errors ----
static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

static cosmo_status fail(cosmo_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CU(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(COSMO_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                            \
  } while (0)

#define TRY(expr)                     \
  do {                                \
    cosmo_status s_ = (expr);         \
    if (s_ != COSMO_OK) return s_;    \
  } while (0)

static int grid_for(int64_t work, int threads, int cap = 148 * 16) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

static int64_t svec_rows(int64_t p) { return p * (p + 1) / 2; }
static int64_t cone_rows(const cosmo_cone& c) {
  return c.type == COSMO_CONE_PSD ? svec_rows(c.dim) : (int64_t)c.dim;
}

// --------------------------------------------------------- validation ---
static cosmo_status validate(const cosmo_problem* pr) {
  if (!pr) return fail(COSMO_E_INVAL, "problem is NULL");
  if (pr->ninst < 1) return fail(COSMO_E_INVAL, "ninst must be >= 1");
  if (!pr->col_off || !pr->row_off || !pr->A_rowptr || !pr->cone_count || !pr->q || !pr->b)
    return fail(COSMO_E_INVAL, "required problem array is NULL");
  const int32_t ni = pr->ninst;
  if (pr->col_off[0] != 0 || pr->row_off[0] != 0)
    return fail(COSMO_E_INVAL, "col_off[0] and row_off[0] must be 0");
  for (int32_t i = 0; i < ni; ++i) {
    if (pr->col_off[i + 1] < pr->col_off[i] || pr->row_off[i + 1] < pr->row_off[i])
      return fail(COSMO_E_INVAL, "offsets of instance %d decrease", i);
    if (pr->cone_count[i] < 0) return fail(COSMO_E_INVAL, "negative cone count");
  }
  const int64_t n = pr->col_off[ni], m = pr->row_off[ni];
  if (n > INT32_MAX || m > INT32_MAX) return fail(COSMO_E_INVAL, "n or m exceeds int32 indexing");
  // A: CSR bounds and block-diagonal structure
  if (pr->A_rowptr[0] != 0) return fail(COSMO_E_INVAL, "A_rowptr[0] != 0");
  int64_t nnzA = pr->A_rowptr[m];
  if (nnzA < 0) return fail(COSMO_E_INVAL, "bad A nnz");
  if (nnzA > 0 && (!pr->A_col || !pr->A_val)) return fail(COSMO_E_INVAL, "A_col/A_val NULL");
  for (int32_t i = 0; i < ni; ++i) {
    for (int64_t r = pr->row_off[i]; r < pr->row_off[i + 1]; ++r) {
      if (pr->A_rowptr[r + 1] < pr->A_rowptr[r]) return fail(COSMO_E_INVAL, "A_rowptr decreases at row %lld", (long long)r);
      for (int64_t e = pr->A_rowptr[r]; e < pr->A_rowptr[r + 1]; ++e) {
        const int64_t c = pr->A_col[e];
        if (c < pr->col_off[i] || c >= pr->col_off[i + 1])
          return fail(COSMO_E_INVAL, "A row %lld references column %lld outside instance %d", (long long)r, (long long)c, i);
        if (!std::isfinite(pr->A_val[e])) return fail(COSMO_E_INVAL, "non-finite A value");
      }
    }
  }
  if (pr->P_rowptr) {
    if (pr->P_rowptr[0] != 0) return fail(COSMO_E_INVAL, "P_rowptr[0] != 0");
    const int64_t nnzP = pr->P_rowptr[n];
    if (nnzP > 0 && (!pr->P_col || !pr->P_val)) return fail(COSMO_E_INVAL, "P_col/P_val NULL");
    for (int32_t i = 0; i < ni; ++i)
      for (int64_t j = pr->col_off[i]; j < pr->col_off[i + 1]; ++j) {
        if (pr->P_rowptr[j + 1] < pr->P_rowptr[j]) return fail(COSMO_E_INVAL, "P_rowptr decreases");
        for (int64_t e = pr->P_rowptr[j]; e < pr->P_rowptr[j + 1]; ++e) {
          const int64_t c = pr->P_col[e];
          if (c < pr->col_off[i] || c >= pr->col_off[i + 1])
            return fail(COSMO_E_INVAL, "P row %lld references column %lld outside instance %d", (long long)j, (long long)c, i);
          if (!std::isfinite(pr->P_val[e])) return fail(COSMO_E_INVAL, "non-finite P value");
        }
      }
  }
  for (int64_t j = 0; j < n; ++j)
    if (!std::isfinite(pr->q[j])) return fail(COSMO_E_INVAL, "non-finite q");
  for (int64_t r = 0; r < m; ++r)
    if (!std::isfinite(pr->b[r])) return fail(COSMO_E_INVAL, "non-finite b");
  // cones
  int64_t ci = 0;
  bool has_box = false;
  for (int32_t i = 0; i < ni; ++i) {
    int64_t rows = 0;
    for (int32_t c = 0; c < pr->cone_count[i]; ++c, ++ci) {
      if (!pr->cones) return fail(COSMO_E_INVAL, "cones NULL");
      const cosmo_cone& cn = pr->cones[ci];
      if (cn.type < COSMO_CONE_ZERO || cn.type > COSMO_CONE_PSD)
        return fail(COSMO_E_INVAL, "unknown cone type %d", cn.type);
      if (cn.dim < 1) return fail(COSMO_E_INVAL, "cone dimension must be >= 1");
      if (cn.type == COSMO_CONE_PSD && cn.dim > 1024) return fail(COSMO_E_INVAL, "PSD order above 1024");
      if (cn.type == COSMO_CONE_BOX) has_box = true;
      rows += cone_rows(cn);
    }
    if (rows != pr->row_off[i + 1] - pr->row_off[i])
      return fail(COSMO_E_INVAL, "cones of instance %d cover %lld rows, instance has %lld", i,
                  (long long)rows, (long long)(pr->row_off[i + 1] - pr->row_off[i]));
  }
  if (has_box) {
    if (!pr->box_l || !pr->box_u) return fail(COSMO_E_INVAL, "box cone without bounds");
    ci = 0;
    for (int32_t i = 0; i < ni; ++i) {
      int64_t r = pr->row_off[i];
      for (int32_t c = 0; c < pr->cone_count[i]; ++c, ++ci) {
        const cosmo_cone& cn = pr->cones[ci];
        const int64_t k = cone_rows(cn);
        if (cn.type == COSMO_CONE_BOX)
          for (int64_t t = r; t < r + k; ++t)
            if (!(pr->box_l[t] <= pr->box_u[t])) return fail(COSMO_E_INVAL, "box bound l > u at row %lld", (long long)t);
        r += k;
      }
    }
  }
  return COSMO_OK;
}

// --------------------------------------------------------- allocation ---
// Device buffers of a batch.  Either owned (one cudaMalloc each), carved
// from caller-owned memory (set_external: 256-byte aligned pieces, nothing
// allocated), or only measured (set_measure: the bytes carving would need).
struct DevArena {
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  unsigned char* ext = nullptr;   // caller memory being carved
  size_t ext_cap = 0, ext_used = 0;
  bool measure = false;
  ~DevArena() { release(); }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
    ext_used = 0;
  }
  void set_external(void* base, size_t cap) { release(); ext = (unsigned char*)base; ext_cap = cap; measure = false; }
  void set_owned() { release(); ext = nullptr; ext_cap = 0; measure = false; }
  void set_measure() { release(); ext = nullptr; ext_cap = 0; measure = true; }
  template <class X>
  cosmo_status alloc(X** out, int64_t count) {
    *out = nullptr;
    if (count <= 0) return COSMO_OK;
    if (measure || ext) {
      const size_t off = (ext_used + 255) & ~(size_t)255, need = (size_t)count * sizeof(X);
      ext_used = off + need;
      bytes = (int64_t)ext_used;
      if (measure) return COSMO_OK;
      if (ext_used > ext_cap)
        return fail(COSMO_E_INVAL, "workspace of %zu bytes too small (%zu needed)", ext_cap, ext_used);
      *out = reinterpret_cast<X*>(ext + off);
      return COSMO_OK;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, (size_t)count * sizeof(X));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(COSMO_E_NOMEM, "cudaMalloc of %lld bytes failed: %s",
                  (long long)(count * (int64_t)sizeof(X)), cudaGetErrorString(e));
    }
    ptrs.push_back(p);
    bytes += count * (int64_t)sizeof(X);
    *out = reinterpret_cast<X*>(p);
    return COSMO_OK;
  }
  template <class X>
  cosmo_status upload(X** out, const std::vector<X>& h) {
    TRY(alloc(out, (int64_t)h.size()));
    if (!h.empty()) CU(cudaMemcpy(*out, h.data(), h.size() * sizeof(X), cudaMemcpyHostToDevice));
    return COSMO_OK;
  }
};

// ------------------------------------------------------ host structure ---
struct HostPlan {
  int32_t ninst = 0;
  int64_t n = 0, m = 0;
  std::vector<int64_t> col_off, row_off;
  std::vector<int32_t> row_inst, col_inst;
  std::vector<uint8_t> row_kind;
  std::vector<int64_t> A_rp, AT_rp, P_rp;
  std::vector<int32_t> A_ci, AT_ci, P_ci;
  std::vector<double> A_v, AT_v, P_v, Pdiag, q, b, bl, bu;
  bool has_P = false, has_box = false;
  std::vector<int64_t> soc_row0; std::vector<int32_t> soc_dim;
  std::vector<int64_t> psd_row0, psd_loff, psd_uoff; std::vector<int32_t> psd_p, psd_sched;
  std::vector<int64_t> rect_row0; std::vector<int32_t> rect_rows;
  std::vector<int32_t> inst_sched;
  std::vector<uint8_t> diag_inst;
  std::vector<int32_t> cg_sched;
  int32_t cg_nt = 256;      // threads of a CG CTA
  int64_t cg_vec = 0;       // max over CG instances of 5 n_i + m_i (reals of the shared-memory CG)
  int32_t cg_cs = 1;        // CTAs per instance (thread-block cluster) in the CG
  bool cg_small = false;    // every CG instance small: n_i + m_i <= 4096, nnz(A_i) + nnz(P_i) <= 16384
                            // (the autotuner then also times one warp per instance)
  int64_t sum_p = 0, sum_p2 = 0;
  int32_t max_p = 0;
};

static void build_plan(const cosmo_problem* pr, HostPlan& h) {
  const int32_t ni = pr->ninst;
  h.ninst = ni;
  h.n = pr->col_off[ni];
  h.m = pr->row_off[ni];
  h.col_off.assign(pr->col_off, pr->col_off + ni + 1);
  h.row_off.assign(pr->row_off, pr->row_off + ni + 1);
  h.row_inst.resize(h.m);
  h.col_inst.resize(h.n);
  for (int32_t i = 0; i < ni; ++i) {
    for (int64_t r = h.row_off[i]; r < h.row_off[i + 1]; ++r) h.row_inst[r] = i;
    for (int64_t j = h.col_off[i]; j < h.col_off[i + 1]; ++j) h.col_inst[j] = i;
  }
  // A and its transpose (stable counting sort by column: entries of each A'
  // row come in increasing row order)
  const int64_t nnzA = pr->A_rowptr[h.m];
  h.A_rp.assign(pr->A_rowptr, pr->A_rowptr + h.m + 1);
  h.A_ci.assign(pr->A_col, pr->A_col + nnzA);
  h.A_v.assign(pr->A_val, pr->A_val + nnzA);
  h.AT_rp.assign(h.n + 1, 0);
  for (int64_t e = 0; e < nnzA; ++e) h.AT_rp[h.A_ci[e] + 1]++;
  for (int64_t j = 0; j < h.n; ++j) h.AT_rp[j + 1] += h.AT_rp[j];
  h.AT_ci.resize(nnzA);
  h.AT_v.resize(nnzA);
  {
    std::vector<int64_t> pos(h.AT_rp.begin(), h.AT_rp.end() - 1);
    for (int64_t r = 0; r < h.m; ++r)
      for (int64_t e = h.A_rp[r]; e < h.A_rp[r + 1]; ++e) {
        const int64_t c = h.A_ci[e];
        h.AT_ci[pos[c]] = (int32_t)r;
        h.AT_v[pos[c]] = h.A_v[e];
        pos[c]++;
      }
  }
  h.Pdiag.assign(h.n, 0.0);
  if (pr->P_rowptr && pr->P_rowptr[h.n] > 0) {
    h.has_P = true;
    const int64_t nnzP = pr->P_rowptr[h.n];
    h.P_rp.assign(pr->P_rowptr, pr->P_rowptr + h.n + 1);
    h.P_ci.assign(pr->P_col, pr->P_col + nnzP);
    h.P_v.assign(pr->P_val, pr->P_val + nnzP);
    for (int64_t j = 0; j < h.n; ++j)
      for (int64_t e = h.P_rp[j]; e < h.P_rp[j + 1]; ++e)
        if (h.P_ci[e] == j) h.Pdiag[j] += h.P_v[e];
  }
  h.q.assign(pr->q, pr->q + h.n);
  h.b.assign(pr->b, pr->b + h.m);
  // cones
  h.row_kind.resize(h.m);
  int64_t ci = 0;
  for (int32_t i = 0; i < ni; ++i) {
    int64_t r = h.row_off[i];
    for (int32_t c = 0; c < pr->cone_count[i]; ++c, ++ci) {
      const cosmo_cone& cn = pr->cones[ci];
      const int64_t k = cone_rows(cn);
      for (int64_t t = r; t < r + k; ++t) h.row_kind[t] = (uint8_t)cn.type;
      if (cn.type == COSMO_CONE_BOX) h.has_box = true;
      if (cn.type == COSMO_CONE_SOC) {
        h.soc_row0.push_back(r);
        h.soc_dim.push_back(cn.dim);
      }
      if (cn.type == COSMO_CONE_PSD) {
        h.psd_row0.push_back(r);
        h.psd_p.push_back(cn.dim);
        h.psd_loff.push_back(h.sum_p);
        h.psd_uoff.push_back(h.sum_p2);
        h.sum_p += cn.dim;
        h.sum_p2 += (int64_t)cn.dim * cn.dim;
        h.max_p = std::max(h.max_p, cn.dim);
      }
      if (cn.type == COSMO_CONE_SOC || cn.type == COSMO_CONE_PSD) {
        h.rect_row0.push_back(r);
        h.rect_rows.push_back((int32_t)k);
      }
      r += k;
    }
  }
  if (h.has_box) {
    h.bl.assign(pr->box_l, pr->box_l + h.m);
    h.bu.assign(pr->box_u, pr->box_u + h.m);
  }
  // schedules: largest PSD blocks first; instances with the most work first
  h.psd_sched.resize(h.psd_p.size());
  std::iota(h.psd_sched.begin(), h.psd_sched.end(), 0);
  std::stable_sort(h.psd_sched.begin(), h.psd_sched.end(),
                   [&](int a, int b) { return h.psd_p[a] > h.psd_p[b]; });
  std::vector<int64_t> work(ni);
  for (int32_t i = 0; i < ni; ++i)
    work[i] = (h.A_rp[h.row_off[i + 1]] - h.A_rp[h.row_off[i]]) * 2 +
              (h.has_P ? h.P_rp[h.col_off[i + 1]] - h.P_rp[h.col_off[i]] : 0) +
              (h.col_off[i + 1] - h.col_off[i]) + (h.row_off[i + 1] - h.row_off[i]);
  h.inst_sched.resize(ni);
  std::iota(h.inst_sched.begin(), h.inst_sched.end(), 0);
  std::stable_sort(h.inst_sched.begin(), h.inst_sched.end(),
                   [&](int a, int b) { return work[a] > work[b]; });
  // diagonal M: P diagonal and no row of A with two nonzeros in distinct columns
  h.diag_inst.assign(ni, 1);
  for (int32_t i = 0; i < ni; ++i) {
    bool d = true;
    for (int64_t r = h.row_off[i]; d && r < h.row_off[i + 1]; ++r)
      if (h.A_rp[r + 1] - h.A_rp[r] > 1) d = false;
    if (h.has_P)
      for (int64_t j = h.col_off[i]; d && j < h.col_off[i + 1]; ++j)
        for (int64_t e = h.P_rp[j]; e < h.P_rp[j + 1]; ++e)
          if (h.P_ci[e] != j && h.P_v[e] != 0.0) { d = false; break; }
    h.diag_inst[i] = d ? 1 : 0;
  }
  int64_t cg_max = 0;
  for (int32_t i : h.inst_sched)
    if (!h.diag_inst[i]) {
      h.cg_sched.push_back(i);
      cg_max = std::max(cg_max, (h.row_off[i + 1] - h.row_off[i]) + (h.col_off[i + 1] - h.col_off[i]));
      h.cg_vec = std::max(h.cg_vec, 5 * (h.col_off[i + 1] - h.col_off[i]) + (h.row_off[i + 1] - h.row_off[i]));
    }
  h.cg_small = !h.cg_sched.empty();
  for (int32_t i : h.cg_sched) {
    const int64_t nz = (h.A_rp[h.row_off[i + 1]] - h.A_rp[h.row_off[i]]) +
                       (h.has_P ? h.P_rp[h.col_off[i + 1]] - h.P_rp[h.col_off[i]] : 0);
    if ((h.row_off[i + 1] - h.row_off[i]) + (h.col_off[i + 1] - h.col_off[i]) > 4096 || nz > 16384)
      h.cg_small = false;
  }
  // large instances take 512-thread CG CTAs (more rows in flight per SpMV);
  // many small ones 256 (two CTAs resident per SM), the smallest (fewer than
  // 1024 rows + columns) 128: fewer warps behind every barrier and reduction
  h.cg_nt = cg_max >= 8192 ? 512 : (cg_max < 1024 ? 128 : 256);
  // few large instances: a cluster of 2 or 4 CTAs per instance, so that the
  // CG of e.g. 64 SOCP instances spreads over more than 64 SMs
  const int64_t ncg = (int64_t)h.cg_sched.size();
  h.cg_cs = 1;
  if (cg_max >= 8192 && ncg > 0) {
    if (4 * ncg <= 148) h.cg_cs = 4;
    else if (2 * ncg <= 148) h.cg_cs = 2;
  }
}

// ------------------------------------------------------- implementation ---
struct Impl {
  virtual ~Impl() {}
  virtual cosmo_status forward(int32_t K, const double* sigma, const void* rho, const void* alpha,
                               const void* x0, const void* s0, const void* y0, void* xK, void* sK,
                               void* yK, double* loss, int32_t tape, cudaStream_t st) = 0;
  virtual cosmo_status backward(const void* gx, const void* gs, const void* gy, const double* gl,
                                void* grho, void* galpha, void* gx0, void* gs0, void* gy0,
                                cudaStream_t st) = 0;
  virtual cosmo_status residuals(const void* x, const void* s, const void* y, double* rp2,
                                 double* rd2, double* obj, cudaStream_t st) = 0;
  virtual cosmo_status solve(const cosmo_solve_params& p, void* x, void* s, void* y, int32_t* iters,
                             double* rbp, double* rbd, double* rho, cudaStream_t st) = 0;
  virtual cosmo_status pol_forward(int32_t K, const double* sigma, const void* tr, const void* ta,
                                   const void* l0, const void* x0, const void* s0, const void* y0, void* xK,
                                   void* sK, void* yK, double* loss, int32_t tape, cudaStream_t st) = 0;
  virtual cosmo_status pol_backward(const void* gx, const void* gs, const void* gy, const double* gl, void* gtr,
                                    void* gta, void* gl0, void* gx0, void* gs0, void* gy0, cudaStream_t st) = 0;
  virtual cosmo_status pol_schedule(void* rho, void* alpha, cudaStream_t st) = 0;
  virtual cosmo_status ws_forward(const void* tx, const void* tc, void* x0, void* s0, void* y0,
                                  cudaStream_t st) = 0;
  virtual cosmo_status ws_backward(const void* tx, const void* tc, const void* gx0, const void* gs0,
                                   const void* gy0, void* gtx, void* gtc, cudaStream_t st) = 0;
  virtual cosmo_status rho_from_log(int32_t K, const double* lr, double eq, void* rho,
                                    cudaStream_t st) = 0;
  virtual cosmo_status rho_from_log_bwd(int32_t K, const void* rho, const void* grho,
                                        double* glog, cudaStream_t st) = 0;
  virtual cosmo_status alpha_bcast(int32_t K, const double* a, void* alpha, cudaStream_t st) = 0;
  virtual cosmo_status alpha_reduce(int32_t K, const void* ga, double* gk, cudaStream_t st) = 0;
  virtual cosmo_status flags_sync(int32_t* out) = 0;
  virtual void info(cosmo_batch_info* o) const = 0;
  virtual cosmo_status profile_enable(const char* tag) = 0;
  virtual cosmo_status profile_read(const char* tag, double* ms, int64_t* n, int32_t reset) = 0;
  virtual size_t real_size() const = 0;
  virtual void get_tuning(cosmo_tuning* t) const = 0;
  virtual cosmo_status tape_eigen(int32_t k, void* lam, void* U, cudaStream_t st) = 0;
  virtual size_t workspace_bytes(int32_t K) = 0;
  virtual cosmo_status set_workspace_ext(int32_t K, void* ws, size_t bytes) = 0;
  virtual cosmo_status set_tuning(const cosmo_tuning& t) = 0;
};

// device staging of cosmo_step_host, owned by the batch so repeated steps
// allocate nothing
struct HostStepBufs {
  int32_t K = 0;
  DevArena a;
  double *lr = nullptr, *ak = nullptr, *glr = nullptr, *gak = nullptr, *loss = nullptr,
         *gloss = nullptr;
  void *rho = nullptr, *alpha = nullptr, *grho = nullptr, *galpha = nullptr;
  void *x0 = nullptr, *s0 = nullptr, *y0 = nullptr, *gx0 = nullptr, *gs0 = nullptr, *gy0 = nullptr;
};

struct cosmo_batch {
  cosmo_options opt;
  HostPlan plan;
  std::unique_ptr<Impl> impl;
  std::unique_ptr<HostStepBufs> hostbufs;
};

// Instantiations of the compile-time-geometry Jacobi (k_psd_fwd_jt2): size
// classes PMAX = 32, 56, 80 at CTA sizes 128..1024 where a thread's work fits
// its registers (at most three tiles and two eigenvector chunks per thread).
template <class T, int PMAX, int NT>
struct Jt2Cfg {
  using G = Jt2Geo<T, PMAX>;
  static constexpr bool room = NT > 32 * G::PW;
  static constexpr int TI = room ? G::items_t(NT) : 1;
  static constexpr int CI = room ? G::items_c(NT) : 1;
  // FP64 items take twice the registers: fewer per thread (no spills at 64 registers)
  static constexpr bool ok = room && (sizeof(T) == 4 ? (TI <= 3 && CI <= 2) : (TI <= 2 && CI <= 1));
};
inline int jt2_pmax(int p) { return p <= 8 ? 8 : (p <= 16 ? 16 : (p <= 32 ? 32 : (p <= 56 ? 56 : (p <= 80 ? 80 : 0)))); }
template <class T, class F>
inline void jt2_for(int pmax, int nt, F f) {   // f(Jt2Cfg) for the (pmax, nt) instantiation, if it exists
#define COSMO_JT2_CASE(PM_, NT_) \
  if (pmax == PM_ && nt == NT_) { if constexpr (Jt2Cfg<T, PM_, NT_>::ok) f(Jt2Cfg<T, PM_, NT_>{}, std::integral_constant<int, PM_>{}, std::integral_constant<int, NT_>{}); return; }
  COSMO_JT2_CASE(8, 64) COSMO_JT2_CASE(8, 128) COSMO_JT2_CASE(16, 64) COSMO_JT2_CASE(16, 128)
  COSMO_JT2_CASE(32, 128) COSMO_JT2_CASE(32, 256) COSMO_JT2_CASE(32, 512) COSMO_JT2_CASE(32, 1024)
  COSMO_JT2_CASE(56, 128) COSMO_JT2_CASE(56, 256) COSMO_JT2_CASE(56, 384) COSMO_JT2_CASE(56, 512)
  COSMO_JT2_CASE(56, 1024)
  COSMO_JT2_CASE(80, 128) COSMO_JT2_CASE(80, 256) COSMO_JT2_CASE(80, 384) COSMO_JT2_CASE(80, 512)
  COSMO_JT2_CASE(80, 1024)
#undef COSMO_JT2_CASE
}
template <class T>
inline bool jt2_exists(int pmax, int nt) {
  bool ok = false;
  jt2_for<T>(pmax, nt, [&](auto, auto, auto) { ok = true; });
  return ok;
}

template <class T, class V>
struct ImplT : Impl {
  cosmo_options opt;
  HostPlan& h;
  DevArena arena;   // K-independent
  DevArena tarena;  // K-dependent (tape, staging)
  Prob<T, V> P{};
  cudaStream_t cap = nullptr;
  int32_t* flags = nullptr;
  unsigned long long* stats = nullptr;  // [6]: Jacobi sweeps, blocks; CG iters, solves; adjoint CG iters, solves
  // K-independent workspace
  T *xi = nullptr, *cg_r = nullptr, *cg_p = nullptr, *cg_u = nullptr, *cg_t = nullptr;
  T *xb[2] = {nullptr, nullptr}, *sb[2] = {nullptr, nullptr}, *yb[2] = {nullptr, nullptr};
  T *gproj = nullptr, *vbar = nullptr, *adjrhs = nullptr, *lamt = nullptr, *rp = nullptr,
    *rd = nullptr;
  double *loss_buf = nullptr, *gloss_buf = nullptr;
  // log-residual meta-loss (loss_kind 1): ||r_d^k||^2, ||r_p^k||^2 for k = 0..K
  // ([K + 1][ninst], tape arena), per-instance weights of one state's cotangent
  double *lr_rd2 = nullptr, *lr_rp2 = nullptr;
  T *lr_wa = nullptr, *lr_wb = nullptr;
  bool lr_track = false;   // forward: store each new state's residual norms
  T *gx_in = nullptr, *gs_in = nullptr, *gy_in = nullptr;
  // tape (segment buffers) and per-step parameters
  int32_t K = 0, cK = 0, nseg = 0, seg_in_buffer = -1;
  bool tape_valid = false, loss_valid = false;
  T *xs = nullptr, *ss = nullptr, *ys = nullptr;        // (cK+1) states
  T *xts = nullptr, *sts = nullptr, *lams = nullptr, *Us = nullptr;  // cK slots
  T *ck_x = nullptr, *ck_s = nullptr, *ck_y = nullptr, *ck_xt = nullptr;  // nseg
  T* ck_U = nullptr;  // nseg x sum p^2: eigenvectors that warm-start each segment
  T *rho_in = nullptr, *rho_rect = nullptr, *dinv = nullptr, *alpha_in = nullptr;
  T *grho_all = nullptr, *galpha_all = nullptr;
  double* sigma_dev = nullptr;
  std::vector<double> sigma_h;
  // graphs
  cudaGraphExec_t gfwd = nullptr, gbwd = nullptr;
  int32_t gfwd_key[3] = {-1, -1, -1};
  std::vector<double> gfwd_sigma, gbwd_sigma;
  int64_t gfwd_nk = 0, gbwd_nk = 0;
  int64_t launched = 0;
  int64_t seq_kernels = 0;  // kernels enqueued by the sequence being built
  // PSD blocks (sorted by p, largest first) split into size buckets, each
  // launched with its own CTA size on a forked stream
  // method 0: CTA-resident Jacobi + shared-memory DK; method 1 (large blocks):
  // tridiagonal + QL in the tape slot + global-memory DK
  // fnt / tpt / variant: CTA size, per-thread work bound and Jacobi kernel of the forward
  struct Bucket { int start, count, maxp, nt; cudaStream_t s; cudaEvent_t done; bool warm_fits; int method;
                  int fnt, tpt, variant; };
  T* dk_work = nullptr;  // 2 x sum p^2: DK scratch of large blocks
  std::vector<Bucket> buckets;
  cudaEvent_t ev_fork = nullptr;
  // optional CUDA-event timing of launches (direct mode only)
  int prof_mode = 0;            // 0 off, 1 every kernel, 2 kernels whose tag == prof_tag
  std::string prof_tag;
  bool capturing = false;
  // graph: the events are nodes of a recorded CUDA graph (recorded again at
  // every replay; collected after each replay, never returned to the pool)
  struct Rec { const char* tag; cudaEvent_t e0, e1; bool graph; };
  std::vector<Rec> prof_pending;
  std::vector<Rec> cap_recs, gfwd_recs, gbwd_recs;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<std::string, std::pair<double, int64_t>>> prof_acc;

  explicit ImplT(const cosmo_options& o, HostPlan& hp) : opt(o), h(hp) {}
  ~ImplT() override {
    if (sv_run_h) cudaFreeHost(sv_run_h);
    for (auto& bk : buckets) { if (bk.s) cudaStreamDestroy(bk.s); if (bk.done) cudaEventDestroy(bk.done); }
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (auto& r : prof_pending) if (!r.graph) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    for (auto* v : {&gfwd_recs, &gbwd_recs})
      for (auto& r : *v) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    for (auto e : ev_pool) cudaEventDestroy(e);
    if (gfwd) cudaGraphExecDestroy(gfwd);
    if (gbwd) cudaGraphExecDestroy(gbwd);
    if (cap) cudaStreamDestroy(cap);
  }
  size_t real_size() const override { return sizeof(T); }

  template <class X>
  static std::vector<X> conv(const std::vector<double>& v) {
    std::vector<X> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (X)v[i];
    return o;
  }
  static std::vector<__nv_bfloat16> conv_bf16(const std::vector<double>& v) {
    std::vector<__nv_bfloat16> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = __float2bfloat16((float)v[i]);
    return o;
  }
  std::vector<V> convV(const std::vector<double>& v) {
    if constexpr (std::is_same<V, __nv_bfloat16>::value) return conv_bf16(v);
    else return conv<V>(v);
  }

  cosmo_status init() {
    CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int64_t *col_off, *row_off, *A_rp, *AT_rp, *P_rp = nullptr, *soc_row0, *psd_row0, *psd_loff,
        *psd_uoff, *rect_row0;
    int32_t *row_inst, *col_inst, *A_ci, *AT_ci, *P_ci = nullptr, *soc_dim, *psd_p, *psd_sched,
        *rect_rows, *inst_sched;
    uint8_t* row_kind;
    V *A_v, *AT_v;
    T *P_v = nullptr, *Pdiag, *q, *b, *bl = nullptr, *bu = nullptr;
    TRY(arena.upload(&col_off, h.col_off));
    TRY(arena.upload(&row_off, h.row_off));
    TRY(arena.upload(&row_inst, h.row_inst));
    TRY(arena.upload(&col_inst, h.col_inst));
    TRY(arena.upload(&row_kind, h.row_kind));
    TRY(arena.upload(&A_rp, h.A_rp));
    TRY(arena.upload(&A_ci, h.A_ci));
    TRY(arena.upload(&A_v, convV(h.A_v)));
    TRY(arena.upload(&AT_rp, h.AT_rp));
    TRY(arena.upload(&AT_ci, h.AT_ci));
    TRY(arena.upload(&AT_v, convV(h.AT_v)));
    if (h.has_P) {
      TRY(arena.upload(&P_rp, h.P_rp));
      TRY(arena.upload(&P_ci, h.P_ci));
      TRY(arena.upload(&P_v, conv<T>(h.P_v)));
    }
    TRY(arena.upload(&Pdiag, conv<T>(h.Pdiag)));
    TRY(arena.upload(&q, conv<T>(h.q)));
    TRY(arena.upload(&b, conv<T>(h.b)));
    if (h.has_box) {
      TRY(arena.upload(&bl, conv<T>(h.bl)));
      TRY(arena.upload(&bu, conv<T>(h.bu)));
    }
    TRY(arena.upload(&soc_row0, h.soc_row0));
    TRY(arena.upload(&soc_dim, h.soc_dim));
    TRY(arena.upload(&psd_row0, h.psd_row0));
    TRY(arena.upload(&psd_p, h.psd_p));
    TRY(arena.upload(&psd_loff, h.psd_loff));
    TRY(arena.upload(&psd_uoff, h.psd_uoff));
    TRY(arena.upload(&psd_sched, h.psd_sched));
    TRY(arena.upload(&rect_row0, h.rect_row0));
    TRY(arena.upload(&rect_rows, h.rect_rows));
    TRY(arena.upload(&inst_sched, h.inst_sched));
    uint8_t* diag_inst;
    int32_t* cg_sched = nullptr;
    TRY(arena.upload(&diag_inst, h.diag_inst));
    TRY(arena.upload(&cg_sched, h.cg_sched));
    P.ninst = h.ninst;
    P.n_total = h.n;
    P.m_total = h.m;
    P.col_off = col_off; P.row_off = row_off; P.row_inst = row_inst; P.col_inst = col_inst;
    P.row_kind = row_kind;
    P.A_rp = A_rp; P.A_ci = A_ci; P.A_v = A_v;
    P.AT_rp = AT_rp; P.AT_ci = AT_ci; P.AT_v = AT_v;
    P.P_rp = P_rp; P.P_ci = P_ci; P.P_v = P_v;
    P.Pdiag = Pdiag; P.q = q; P.b = b; P.box_l = bl; P.box_u = bu;
    P.nsoc = (int32_t)h.soc_row0.size(); P.soc_row0 = soc_row0; P.soc_dim = soc_dim;
    P.npsd = (int32_t)h.psd_p.size(); P.psd_row0 = psd_row0; P.psd_p = psd_p;
    P.psd_loff = psd_loff; P.psd_uoff = psd_uoff; P.psd_sched = psd_sched;
    P.nrect = (int32_t)h.rect_row0.size(); P.rect_row0 = rect_row0; P.rect_rows = rect_rows;
    P.inst_sched = inst_sched;
    P.diag_inst = diag_inst;
    P.n_cg = (int32_t)h.cg_sched.size();
    P.cg_sched = cg_sched;
    const int64_t n = h.n, m = h.m;
    TRY(arena.alloc(&flags, h.ninst));
    CU(cudaMemset(flags, 0, sizeof(int32_t) * h.ninst));
    TRY(arena.alloc(&stats, 6));
    CU(cudaMemset(stats, 0, sizeof(unsigned long long) * 6));
    TRY(arena.alloc(&xi, n)); TRY(arena.alloc(&cg_r, n)); TRY(arena.alloc(&cg_p, n));
    TRY(arena.alloc(&cg_u, n)); TRY(arena.alloc(&cg_t, m));
    // the shared-memory CG may take up to CG_SMEM_MAX bytes (set outside any graph capture)
    CU(cudaFuncSetAttribute(k_pcg_smem<T, V, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG_SMEM_MAX));
    CU(cudaFuncSetAttribute(k_pcg_local<T, V, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG_SMEM_MAX));
    CU(cudaFuncSetAttribute(k_pcg_smem<T, V, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG_SMEM_MAX));
    CU(cudaFuncSetAttribute(k_pcg_smem<T, V, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG_SMEM_MAX));
    CU(cudaFuncSetAttribute(k_pcg_local<T, V, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG_SMEM_MAX));
    CU(cudaFuncSetAttribute(k_pcg_local<T, V, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG_SMEM_MAX));
    if constexpr (std::is_same<T, float>::value)   // tensor-core weight sums: 48 KB + the padded layout
      CU(cudaFuncSetAttribute(k_ws_atb_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws_tc_smem(64)));
    // shared memory of the CG with the instance's matrices staged too (largest CG instance)
    cg_local = 0;
    for (int32_t i : h.cg_sched) {
      const int64_t ni = h.col_off[i + 1] - h.col_off[i], mi = h.row_off[i + 1] - h.row_off[i];
      const int64_t nnzA = h.A_rp[h.row_off[i + 1]] - h.A_rp[h.row_off[i]];
      size_t b = ((sizeof(T) * (5 * ni + mi) + 15) & ~(size_t)15) + 2 * smem_csr_bytes(std::max(ni, mi), nnzA, sizeof(V));
      if (h.has_P) b += smem_csr_bytes(ni, h.P_rp[h.col_off[i + 1]] - h.P_rp[h.col_off[i]], sizeof(T));
      cg_local = std::max(cg_local, b);
    }
    if (P.n_cg && ((opt.cg_cluster == -1 && cg_smem_bytes() > CG_SMEM_MAX) ||
                   (opt.cg_cluster == -2 && cg_local > CG_SMEM_MAX)))
      return fail(COSMO_E_INVAL, "cg_cluster %d: the CG's shared-memory data (%zu B) exceeds %zu B",
                  opt.cg_cluster, opt.cg_cluster == -1 ? cg_smem_bytes() : cg_local, CG_SMEM_MAX);
    for (int i = 0; i < 2; ++i) {
      TRY(arena.alloc(&xb[i], n)); TRY(arena.alloc(&sb[i], m)); TRY(arena.alloc(&yb[i], m));
    }
    TRY(arena.alloc(&gproj, m)); TRY(arena.alloc(&vbar, m)); TRY(arena.alloc(&adjrhs, n));
    TRY(arena.alloc(&lamt, n)); TRY(arena.alloc(&rp, m)); TRY(arena.alloc(&rd, n));
    TRY(arena.alloc(&gx_in, n)); TRY(arena.alloc(&gs_in, m)); TRY(arena.alloc(&gy_in, m));
    TRY(arena.alloc(&loss_buf, h.ninst)); TRY(arena.alloc(&gloss_buf, h.ninst));
    TRY(arena.alloc(&lr_wa, h.ninst)); TRY(arena.alloc(&lr_wb, h.ninst));
    if (P.npsd > 0) {
      int dev = 0, maxs = 0;
      CU(cudaGetDevice(&dev));
      CU(cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      // Jacobi size classes: p > 56 -> 512 threads, 33..56 -> 256, <= 32 -> 128.
      // Blocks above the cutoff (option eig_jacobi_max_p; by default the
      // largest p whose warm-started Jacobi and DK fit in shared memory) take
      // the large-block path with 256 threads.
      const int variant = opt.eig_variant == 0 || opt.eig_variant == 3 ? 2 : opt.eig_variant;
      auto jt2_ok = [&](int p, int fnt) {
        return jt2_pmax(p) && jt2_exists<T>(jt2_pmax(p), fnt) && (int64_t)jt2_bytes(p, fnt) <= maxs;
      };
      // (blocks of order <= 16 take 64 threads where the compile-time geometry has them)
      auto fwd_threads = [&](int p) {
        if (opt.eig_threads) return opt.eig_threads;
        if (p <= 16 && opt.eig_variant != 1 && opt.eig_variant != 2 && jt2_exists<T>(jt2_pmax(p), 64)) return 64;
        return p > 56 ? 512 : (p > 32 ? 256 : 128);
      };
      auto fits_jacobi = [&](int p) {
        const int nt = p > 56 ? 512 : (p > 32 ? 256 : 128), fnt = fwd_threads(p);
        if ((int64_t)psd_bwd_smem<T>(p, nt) > maxs) return false;
        if (variant == 2) return (int64_t)jt_smem<T>(p, fnt) <= maxs && jt_ipt(p, fnt) <= 8 && p <= 180;
        return (int64_t)psd_fwd_smem_warm<T>(p, fnt) <= maxs;
      };
      auto class_of = [&](int p) {
        const bool big = opt.eig_jacobi_max_p > 0 ? (p > opt.eig_jacobi_max_p || !fits_jacobi(p)) : !fits_jacobi(p);
        if (big) return 1000;                    // large-block path
        return p > 56 ? 512 : (p > 32 ? 256 : 128);
      };
      bool any_big = false;
      for (size_t q = 0; q < h.psd_sched.size();) {
        const int p0 = h.psd_p[h.psd_sched[q]];
        const int cls = class_of(p0);
        size_t e = q;
        while (e < h.psd_sched.size() && class_of(h.psd_p[h.psd_sched[e]]) == cls) ++e;
        const int method = cls == 1000 ? 1 : 0;
        const int nt = method ? 256 : cls;
        const int fnt = method ? 256 : fwd_threads(p0);
        const int bvar = (opt.eig_variant == 0 || opt.eig_variant == 3) && method == 0 && jt2_ok(p0, fnt) ? 3 : variant;
        if (opt.eig_variant == 3 && method == 0 && bvar != 3)
          return fail(COSMO_E_INVAL, "eig_variant 3: no instantiation for order %d with %d threads", p0, fnt);
        Bucket bk{(int)q, (int)(e - q), p0, nt, nullptr, nullptr,
                  method == 0 && (variant == 2 || (int64_t)psd_fwd_smem_warm<T>(p0, fnt) <= (int64_t)maxs), method,
                  fnt, jt_ipt(p0, fnt) <= 2 ? 2 : (jt_ipt(p0, fnt) <= 4 ? 4 : 8), bvar};
        CU(cudaStreamCreateWithFlags(&bk.s, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&bk.done, cudaEventDisableTiming));
        if (method == 0) {
          const size_t fs = bvar == 3 ? jt2_bytes(p0, fnt) : (variant == 2 ? jt_smem<T>(p0, fnt) : psd_fwd_smem<T>(p0, fnt)),
                       bs = psd_bwd_smem<T>(p0, nt);
          if ((int64_t)fs > maxs || (int64_t)bs > maxs)
            return fail(COSMO_E_INVAL, "PSD order %d needs %zu B of shared memory (device allows %d)",
                        p0, std::max(fs, bs), maxs);
        } else {
          any_big = true;
          if ((int64_t)tql_smem<T>(p0, nt) > maxs)
            return fail(COSMO_E_INVAL, "PSD order %d too large", p0);
        }
        // classes of order <= TPB_MAXP in FP32: one block per thread (kernels_tpb.cuh)
        if (std::is_same<T, float>::value && method == 0 && p0 <= TPB_MAXP && opt.eig_variant == 0 &&
            opt.eig_threads == 0) {
          bk.method = 2;
          bk.fnt = TPB_NT;
          bk.warm_fits = true;
        }
        buckets.push_back(bk);
        q = e;
      }
      if (any_big) TRY(arena.alloc(&dk_work, 2 * h.sum_p2));
      smem_max = maxs;
      CU(cudaFuncSetAttribute(k_psd_fwd_tql<T, V, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
      CU(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
      CU(cudaFuncSetAttribute(k_psd_fwd<T, V, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
      CU(cudaFuncSetAttribute(k_psd_fwd<T, V, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
      CU(cudaFuncSetAttribute(k_psd_fwd<T, V, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
#define COSMO_JT_ATTR(NT_, IPT_) \
      CU(cudaFuncSetAttribute(k_psd_fwd_jt<T, V, NT_, IPT_>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs))
      COSMO_JT_ATTR(128, 2); COSMO_JT_ATTR(128, 4); COSMO_JT_ATTR(128, 8);
      COSMO_JT_ATTR(256, 2); COSMO_JT_ATTR(256, 4); COSMO_JT_ATTR(256, 8);
      COSMO_JT_ATTR(512, 2); COSMO_JT_ATTR(512, 4); COSMO_JT_ATTR(512, 8);
      COSMO_JT_ATTR(1024, 2); COSMO_JT_ATTR(1024, 4); COSMO_JT_ATTR(1024, 8);
#undef COSMO_JT_ATTR
      for (int pm : {8, 16, 32, 56, 80})
        for (int nt_ : {64, 128, 256, 384, 512, 1024})
          jt2_for<T>(pm, nt_, [&](auto c, auto pmc, auto ntc) {
            using C = decltype(c);
            if ((int64_t)Jt2Geo<T, decltype(pmc)::value>::bytes(ntc) <= maxs) {
              cudaFuncSetAttribute(k_psd_fwd_jt2<T, V, decltype(ntc)::value, decltype(pmc)::value, C::TI, C::CI>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
              if constexpr (std::is_same<T, float>::value && std::is_same<V, float>::value)
                cudaFuncSetAttribute(k_fwd_persist_jt2<T, V, decltype(ntc)::value, decltype(pmc)::value, C::TI, C::CI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
            }
          });
      CU(cudaGetLastError());
      CU(cudaFuncSetAttribute(k_psd_fwd_tpb<T, V, TPB_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
      CU(cudaFuncSetAttribute(k_psd_bwd_tpb<T, V, TPB_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
      CU(cudaFuncSetAttribute(k_psd_bwd<T, V, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
      CU(cudaFuncSetAttribute(k_psd_bwd<T, V, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
      CU(cudaFuncSetAttribute(k_psd_bwd<T, V, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
      if constexpr (std::is_same<T, float>::value)
        CU(cudaFuncSetAttribute(k_psd_bwd_tc<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dk_tc_smem(DK_TC_MAXP)));
    }
    if (opt.autotune) TRY(tune());
    rect_small = !h.rect_rows.empty();
    for (int32_t nr : h.rect_rows) rect_small = rect_small && nr <= 64;
    // persistent forward (kernels_persist.cuh): FP32 batches (FP32 values)
    // of diagonal instances with exactly one PSD block each and no SOC rows
    if constexpr (std::is_same<T, float>::value && std::is_same<V, float>::value) {
      persist_shape = opt.fwd_persistent == 1 && P.nsoc == 0 && P.n_cg == 0 && h.ninst > 0 &&
                      h.psd_p.size() == (size_t)h.ninst;
      if (persist_shape) {
        std::vector<int32_t> cnt(h.ninst, 0);
        for (int64_t r0 : h.psd_row0) ++cnt[h.row_inst[r0]];
        for (int32_t c : cnt) persist_shape = persist_shape && c == 1;
      }
    }
    return COSMO_OK;
  }
  bool persist_shape = false;
  // every SOC / PSD block has at most 64 rows: the rectification kernels take
  // 8 lanes per block instead of a warp
  bool rect_small = false;
  // the persistent forward applies now: open loop, squared-residual loss,
  // every size class on the compile-time-geometry Jacobi
  bool persist_now() const {
    if (!persist_shape || pol_mode || opt.loss_kind != 0 || buckets.empty()) return false;
    for (const auto& bk : buckets)
      if (bk.method != 0 || bk.variant != 3) return false;
    return true;
  }

  // ------------------------------------------------------------- tuning --
  // Candidate launch configurations are timed with CUDA events on synthetic
  // data of the batch's own shapes (see cosmo_tuning in the header); the
  // choice is cached per process under a key of the device, the types and
  // the shapes.
  int smem_max = 0;
  bool tuned = false;
  double tune_ms = 0.0;
  struct TuneResult { std::vector<int> method, fnt; int cg = 0; };
  static std::mutex& tune_mu() { static std::mutex m; return m; }
  static std::vector<std::pair<std::string, TuneResult>>& tune_cache() {
    static std::vector<std::pair<std::string, TuneResult>> c;
    return c;
  }
  std::string tune_key() const {
    uint64_t hsh = 1469598103934665603ull;   // FNV-1a over the class orders in schedule order
    for (int32_t blk : h.psd_sched) { hsh ^= (uint64_t)h.psd_p[blk]; hsh *= 1099511628211ull; }
    char buf[512];
    snprintf(buf, sizeof buf, "%d|%zu|%zu|%d|%d|%d|%d|%llx|%zu|cg%d,%lld,%zu,%d,%lld,%lld,%lld,%lld", opt.device,
             sizeof(T), sizeof(V), opt.eig_warm_start, opt.dk_tensor_cores, opt.eig_jacobi_max_p, opt.eig_variant,
             (unsigned long long)hsh, buckets.size(), P.n_cg, (long long)h.cg_vec, cg_local, h.cg_nt,
             (long long)h.A_ci.size(), (long long)h.P_ci.size(), (long long)h.n, (long long)h.m);
    return std::string(buf);
  }
  static size_t jt2_bytes(int p, int fnt) {
    size_t b = 0;
    jt2_for<T>(jt2_pmax(p), fnt, [&](auto, auto pmc, auto) { b = Jt2Geo<T, decltype(pmc)::value>::bytes(fnt); });
    return b;
  }
  bool jt2_fits(int p, int fnt) const {
    return jt2_pmax(p) && jt2_exists<T>(jt2_pmax(p), fnt) && (int64_t)jt2_bytes(p, fnt) <= smem_max;
  }
  bool jt_fits(int p, int fnt) const {
    return (fnt == 128 || fnt == 256 || fnt == 512 || fnt == 1024) && fnt > 32 * jt_pair_warps(p) && (int64_t)jt_smem<T>(p, fnt) <= smem_max && jt_ipt(p, fnt) <= 8 && p <= 180;
  }
  bool ql_fits(int p) const { return (int64_t)tql_smem<T>(p, 256) <= smem_max; }
  bool bwd_fits(const Bucket& bk) const {
    if (std::is_same<T, float>::value && opt.dk_tensor_cores && bk.maxp <= DK_TC_MAXP) return true;
    return (int64_t)psd_bwd_smem<T>(bk.maxp, bk.nt) <= smem_max;
  }
  static int ipt_class(int p, int fnt) {
    const int i = jt_ipt(p, fnt);
    return i <= 2 ? 2 : (i <= 4 ? 4 : 8);
  }
  // a class's configuration: method 0 = Jacobi (this batch's variant), 1 = QL,
  // 2 = one block per thread (FP32, orders <= TPB_MAXP)
  cosmo_status config_bucket(Bucket& bk, int method, int fnt) {
    if (method == 2) {
      if (!std::is_same<T, float>::value || bk.maxp > TPB_MAXP)
        return fail(COSMO_E_INVAL, "order %d does not fit the one-block-per-thread path", bk.maxp);
      bk.method = 2;
      bk.fnt = TPB_NT;
      bk.warm_fits = true;
      return COSMO_OK;
    }
    if (method == 1) {
      if (!ql_fits(bk.maxp)) return fail(COSMO_E_INVAL, "order %d does not fit the QL path", bk.maxp);
      if (!dk_work) TRY(arena.alloc(&dk_work, 2 * h.sum_p2));
      bk.method = 1;
      bk.fnt = 256;
      return COSMO_OK;
    }
    const int variant = opt.eig_variant == 0 ? (jt2_fits(bk.maxp, fnt) ? 3 : 2) : opt.eig_variant;
    const bool ok = variant == 3   ? jt2_fits(bk.maxp, fnt)
                    : variant == 2 ? jt_fits(bk.maxp, fnt)
                                   : (fnt <= 512 && fnt >= 128 && (int64_t)psd_fwd_smem_warm<T>(bk.maxp, fnt) <= smem_max);
    Bucket t = bk;
    t.method = 0;
    if (!ok || !bwd_fits(t)) return fail(COSMO_E_INVAL, "order %d does not fit Jacobi with %d threads", bk.maxp, fnt);
    bk.method = 0;
    bk.variant = variant;
    bk.fnt = fnt;
    bk.tpt = ipt_class(bk.maxp, fnt);
    bk.warm_fits = true;
    return COSMO_OK;
  }
  void drop_graphs() {
    if (gfwd) { cudaGraphExecDestroy(gfwd); gfwd = nullptr; }
    if (gbwd) { cudaGraphExecDestroy(gbwd); gbwd = nullptr; }
    release_recs(gfwd_recs);
    release_recs(gbwd_recs);
    gfwd_key[0] = -1;
  }
  cosmo_status apply_tune(const TuneResult& r) {
    for (size_t i = 0; i < buckets.size(); ++i) TRY(config_bucket(buckets[i], r.method[i], r.fnt[i]));
    cg_mode = r.cg;
    drop_graphs();
    return COSMO_OK;
  }
  template <class F>
  float time_min(cudaStream_t st, F fn) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fn();
    float best = 3.0e38f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0, st);
      fn();
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
  }
  cosmo_status tune() {
    const auto t0 = std::chrono::steady_clock::now();
    const std::string key = tune_key();
    {
      std::lock_guard<std::mutex> lk(tune_mu());
      for (auto& e : tune_cache())
        if (e.first == key) {
          TRY(apply_tune(e.second));
          tuned = true;
          tune_ms = 0.0;
          return COSMO_OK;
        }
    }
    TuneResult res;
    cudaStream_t st = nullptr;
    CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cosmo_status status = tune_run(st, res);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (status != COSMO_OK) return status;
    if (e != cudaSuccess) return fail(COSMO_E_CUDA, "tuning: %s", cudaGetErrorString(e));
    TRY(apply_tune(res));
    {
      std::lock_guard<std::mutex> lk(tune_mu());
      tune_cache().push_back(std::make_pair(key, res));
    }
    tuned = true;
    tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return COSMO_OK;
  }
  cosmo_status tune_run(cudaStream_t st, TuneResult& res) {
    DevArena ta;
    res.method.resize(buckets.size());
    res.fnt.resize(buckets.size());
    for (size_t i = 0; i < buckets.size(); ++i) { res.method[i] = buckets[i].method; res.fnt[i] = buckets[i].fnt; }
    res.cg = cg_mode;
    std::mt19937_64 rng(20260613ull);
    std::normal_distribution<double> nd(0.0, 1.0);
    const bool tune_psd = P.npsd > 0 && opt.eig_threads == 0 && opt.eig_variant != 1;
    const bool tune_cg = P.n_cg > 0 && opt.cg_cluster == 0;
    const int64_t m = h.m, n = h.n, ni = h.ninst;
    if (tune_psd) {
      // a random symmetric iterate per block, and a perturbation of it (5%)
      // projected warm-started from the first one's eigenvectors
      std::vector<double> v0(m), v1(m), gv(m);
      for (int64_t r = 0; r < m; ++r) { v0[r] = nd(rng); v1[r] = v0[r] + 0.05 * nd(rng); gv[r] = nd(rng); }
      T *s0, *s1, *zero, *one_r, *one_a, *sn, *yn, *lam, *U0, *U1, *g, *vb;
      int32_t* fl;
      TRY(ta.upload(&s0, conv<T>(v0))); TRY(ta.upload(&s1, conv<T>(v1))); TRY(ta.upload(&g, conv<T>(gv)));
      TRY(ta.upload(&one_r, std::vector<T>(m, T(1)))); TRY(ta.upload(&one_a, std::vector<T>(ni, T(1))));
      TRY(ta.alloc(&zero, m)); TRY(ta.alloc(&sn, m)); TRY(ta.alloc(&yn, m)); TRY(ta.alloc(&vb, m));
      TRY(ta.alloc(&lam, h.sum_p)); TRY(ta.alloc(&U0, h.sum_p2)); TRY(ta.alloc(&U1, h.sum_p2));
      TRY(ta.alloc(&fl, ni));
      CU(cudaMemsetAsync(zero, 0, sizeof(T) * m, st));
      CU(cudaMemsetAsync(fl, 0, sizeof(int32_t) * ni, st));
      const PsdIterIO<T> io0{s0, zero, zero, one_r, one_a, sn, yn, P.row_inst};
      const PsdIterIO<T> io1{s1, zero, zero, one_r, one_a, sn, yn, P.row_inst};
      const PsdBwdIO<T> bio{g, vb, P.row_inst};
      for (size_t i = 0; i < buckets.size(); ++i) {
        const Bucket base = buckets[i];
        psd_fwd_bucket(base, st, io0, lam, U0, nullptr, fl, nullptr);
        CU(cudaGetLastError());
        float best = 3.0e38f;
        float bwd[3] = {-1.f, -1.f, -1.f};
        std::vector<std::pair<int, int>> cands;
        for (int fnt : {64, 128, 256, 384, 512, 1024}) cands.push_back(std::make_pair(0, fnt));
        if (opt.eig_jacobi_max_p == 0 && base.maxp >= 48) cands.push_back(std::make_pair(1, 256));
        if (std::is_same<T, float>::value && opt.eig_variant == 0 && base.maxp <= TPB_MAXP)
          cands.push_back(std::make_pair(2, TPB_NT));
        for (const auto& c : cands) {
          Bucket bk = base;
          if (c.first == 1 ? !ql_fits(bk.maxp)
                           : c.first == 0 && !(jt2_fits(bk.maxp, c.second) || jt_fits(bk.maxp, c.second))) continue;
          if (config_bucket(bk, c.first, c.second) != COSMO_OK) { g_err.clear(); continue; }
          const T* up = bk.method != 1 && opt.eig_warm_start ? U0 : nullptr;
          const float f = time_min(st, [&]() { psd_fwd_bucket(bk, st, io1, lam, U1, up, fl, nullptr); });
          CU(cudaGetLastError());
          if (bwd[bk.method] < 0.f) {
            bwd[bk.method] = time_min(st, [&]() { psd_bwd_bucket(bk, st, bio, lam, U1, fl); });
            CU(cudaGetLastError());
          }
          if (f + bwd[bk.method] < best) {
            best = f + bwd[bk.method];
            res.method[i] = bk.method;
            res.fnt[i] = bk.fnt;
          }
        }
      }
    }
    if (tune_cg) {
      // 20 iterations of the batch's operator, rho = 0.1 (1e2 on zero-cone rows)
      std::vector<double> rh(m), bv(n);
      for (int64_t r = 0; r < m; ++r) rh[r] = h.row_kind[r] == K_ZERO ? 100.0 : 0.1;
      for (int64_t j = 0; j < n; ++j) bv[j] = nd(rng);
      T *rho, *dv, *rhs, *x;
      int32_t* fl;
      double* sig;
      TRY(ta.upload(&rho, conv<T>(rh))); TRY(ta.upload(&rhs, conv<T>(bv)));
      TRY(ta.upload(&sig, std::vector<double>(1, 1e-6)));
      TRY(ta.alloc(&dv, n)); TRY(ta.alloc(&x, n)); TRY(ta.alloc(&fl, ni));
      CU(cudaMemsetAsync(fl, 0, sizeof(int32_t) * ni, st));
      k_precond<T, V><<<grid_for(n, 256), 256, 0, st>>>(P, 1, (const double*)sig, (const T*)rho, dv);
      CgArgs<T> ca{};
      ca.rhs = rhs; ca.x = x; ca.x0 = nullptr; ca.rho = rho; ca.dinv = dv; ca.sigma = 1e-6;
      ca.r = cg_r; ca.p = cg_p; ca.u = cg_u; ca.t = cg_t; ca.tol = 1e-30; ca.maxit = 20; ca.zero_start = 1;
      ca.flag_bit = F_CG_CAP; ca.flags = fl; ca.iters = nullptr; ca.stats = nullptr;
      std::vector<int> cands;
      if (h.cg_small) cands.push_back(-4);
      if (cg_local <= CG_SMEM_MAX) cands.push_back(-2);
      if (cg_smem_bytes() <= CG_SMEM_MAX) cands.push_back(-1);
      cands.push_back(-3);
      cands.push_back(2);
      cands.push_back(4);
      const int keep = cg_mode;
      float best = 3.0e38f;
      for (int c : cands) {
        cg_mode = c;
        const float t = time_min(st, [&]() { launch_pcg("tune", st, ca); });
        CU(cudaGetLastError());
        if (t < best) { best = t; res.cg = c; }
      }
      cg_mode = keep;
    }
    return COSMO_OK;
  }
  cosmo_status tape_eigen(int32_t k, void* lamo, void* Uo, cudaStream_t st) override {
    if (!h.sum_p) return fail(COSMO_E_INVAL, "the batch has no PSD block");
    if (!tape_valid) return fail(COSMO_E_STATE, "no forward with a tape");
    if (k < 0 || k >= K) return fail(COSMO_E_INVAL, "step %d out of range [0, %d)", k, K);
    const int32_t seg = k / cK;
    if (seg != seg_in_buffer) return fail(COSMO_E_STATE, "step %d is not in the segment held in the buffer", k);
    const int64_t sl = k - (int64_t)seg * cK;
    if (lamo) CU(cudaMemcpyAsync(lamo, lams + sl * h.sum_p, sizeof(T) * h.sum_p, cudaMemcpyDeviceToDevice, st));
    if (Uo) CU(cudaMemcpyAsync(Uo, Us + sl * h.sum_p2, sizeof(T) * h.sum_p2, cudaMemcpyDeviceToDevice, st));
    return COSMO_OK;
  }
  void get_tuning(cosmo_tuning* t) const override {
    memset(t, 0, sizeof(*t));
    t->n_classes = (int32_t)std::min<size_t>(buckets.size(), COSMO_MAX_PSD_CLASSES);
    for (int i = 0; i < t->n_classes; ++i) {
      t->class_maxp[i] = buckets[i].maxp;
      t->class_count[i] = buckets[i].count;
      t->class_method[i] = buckets[i].method;
      t->class_threads[i] = buckets[i].fnt;
    }
    t->cg_kernel = opt.cg_cluster != 0 ? opt.cg_cluster : cg_mode;
    t->tuned = tuned ? 1 : 0;
    t->tune_ms = tune_ms;
  }
  cosmo_status set_tuning(const cosmo_tuning& t) override {
    if (t.n_classes != (int32_t)buckets.size() || buckets.size() > COSMO_MAX_PSD_CLASSES)
      return fail(COSMO_E_INVAL, "tuning has %d classes, the batch %zu", t.n_classes, buckets.size());
    for (size_t i = 0; i < buckets.size(); ++i)
      if (t.class_maxp[i] != buckets[i].maxp || t.class_count[i] != buckets[i].count ||
          !(t.class_method[i] == 0 || t.class_method[i] == 1 || t.class_method[i] == 2))
        return fail(COSMO_E_INVAL, "tuning class %zu does not match the batch", i);
    const int cg = t.cg_kernel;
    if (!(cg >= -4 && cg <= 4 && cg != 3) || (cg == -1 && cg_smem_bytes() > CG_SMEM_MAX) ||
        (cg == -2 && cg_local > CG_SMEM_MAX))
      return fail(COSMO_E_INVAL, "tuning: CG kernel %d not available", cg);
    std::vector<Bucket> nb = buckets;
    for (size_t i = 0; i < nb.size(); ++i) TRY(config_bucket(nb[i], t.class_method[i], t.class_threads[i]));
    CU(cudaDeviceSynchronize());
    buckets = nb;
    cg_mode = cg;
    tuned = t.tuned != 0;
    tune_ms = t.tune_ms;
    drop_graphs();
    return COSMO_OK;
  }

  // (re)allocate the tape for K steps with checkpoint interval c
  // caller-owned workspace for the tape of K-step forwards (cosmo_batch_set_workspace)
  void* ws_ext = nullptr;
  size_t ws_ext_bytes = 0;
  int32_t ws_ext_K = 0;
  bool tape_external = false;

  // bytes of the K-step tape and step parameters (what ensure_tape places)
  size_t tape_bytes(int32_t newK) {
    DevArena a;
    a.set_measure();
    TapePtrs t;
    tape_layout(a, newK, opt.checkpoint_every > 0 ? std::min(opt.checkpoint_every, newK) : newK, t);
    return (size_t)a.bytes + 256;   // + alignment of an arbitrary base
  }
  size_t workspace_bytes(int32_t newK) override { return tape_bytes(newK); }
  cosmo_status set_workspace_ext(int32_t newK, void* ws, size_t bytes) override { return set_workspace(newK, ws, bytes); }
  cosmo_status set_workspace(int32_t newK, void* ws, size_t bytes) {
    if (ws) {
      if (newK < 1) return fail(COSMO_E_INVAL, "K must be >= 1");
      if (bytes < tape_bytes(newK))
        return fail(COSMO_E_INVAL, "workspace of %zu bytes, %zu needed for K = %d", bytes, tape_bytes(newK), newK);
    }
    CU(cudaDeviceSynchronize());
    ws_ext = ws;
    ws_ext_bytes = ws ? bytes : 0;
    ws_ext_K = ws ? newK : 0;
    // the next forward lays the tape out again
    drop_graphs();
    tarena.set_owned();
    xs = nullptr;
    K = 0;
    tape_valid = false;
    tape_external = false;
    return COSMO_OK;
  }

  cosmo_status ensure_tape(int32_t newK) {
    int32_t c = opt.checkpoint_every > 0 ? std::min(opt.checkpoint_every, newK) : newK;
    const bool use_ext = ws_ext && ws_ext_K == newK;
    if (newK == K && c == cK && xs && use_ext == tape_external) return COSMO_OK;
    drop_graphs();
    CU(cudaDeviceSynchronize());
    if (use_ext) {
      const uintptr_t base = (reinterpret_cast<uintptr_t>(ws_ext) + 255) & ~uintptr_t(255);
      tarena.set_external(reinterpret_cast<void*>(base), ws_ext_bytes - (size_t)(base - reinterpret_cast<uintptr_t>(ws_ext)));
    } else {
      tarena.set_owned();
    }
    tape_external = use_ext;
    tape_valid = false;
    K = newK;
    cK = c;
    nseg = (K + cK - 1) / cK;
    TapePtrs t;
    TRY(tape_layout(tarena, K, cK, t));
    lr_rd2 = t.lr_rd2; lr_rp2 = t.lr_rp2; sigma_dev = t.sigma_dev;
    xs = t.xs; ss = t.ss; ys = t.ys; xts = t.xts; sts = t.sts; lams = t.lams; Us = t.Us;
    ck_x = t.ck_x; ck_s = t.ck_s; ck_y = t.ck_y; ck_xt = t.ck_xt; ck_U = t.ck_U;
    rho_in = t.rho_in; rho_rect = t.rho_rect; dinv = t.dinv; alpha_in = t.alpha_in;
    grho_all = t.grho_all; galpha_all = t.galpha_all;
    return COSMO_OK;
  }

  struct TapePtrs {
    double *lr_rd2 = nullptr, *lr_rp2 = nullptr, *sigma_dev = nullptr;
    T *xs = nullptr, *ss = nullptr, *ys = nullptr, *xts = nullptr, *sts = nullptr, *lams = nullptr, *Us = nullptr;
    T *ck_x = nullptr, *ck_s = nullptr, *ck_y = nullptr, *ck_xt = nullptr, *ck_U = nullptr;
    T *rho_in = nullptr, *rho_rect = nullptr, *dinv = nullptr, *alpha_in = nullptr, *grho_all = nullptr,
      *galpha_all = nullptr;
  };
  cosmo_status tape_layout(DevArena& ta, int32_t K_, int32_t c_, TapePtrs& t) {
    const int64_t n = h.n, m = h.m, ni = h.ninst;
    const int32_t nseg_ = (K_ + c_ - 1) / c_;
    const int32_t K = K_, cK = c_, nseg = nseg_;
    DevArena& tarena = ta;
    TRY(tarena.alloc(&t.lr_rd2, (int64_t)(K + 1) * ni)); TRY(tarena.alloc(&t.lr_rp2, (int64_t)(K + 1) * ni));
    TRY(tarena.alloc(&t.xs, (cK + 1) * n)); TRY(tarena.alloc(&t.ss, (cK + 1) * m));
    TRY(tarena.alloc(&t.ys, (cK + 1) * m));
    TRY(tarena.alloc(&t.xts, (int64_t)cK * n)); TRY(tarena.alloc(&t.sts, (int64_t)cK * m));
    TRY(tarena.alloc(&t.lams, (int64_t)cK * h.sum_p)); TRY(tarena.alloc(&t.Us, (int64_t)cK * h.sum_p2));
    TRY(tarena.alloc(&t.ck_x, nseg * n)); TRY(tarena.alloc(&t.ck_s, nseg * m));
    TRY(tarena.alloc(&t.ck_y, nseg * m)); TRY(tarena.alloc(&t.ck_xt, nseg * n));
    TRY(tarena.alloc(&t.ck_U, (int64_t)nseg * h.sum_p2));
    TRY(tarena.alloc(&t.rho_in, (int64_t)K * m)); TRY(tarena.alloc(&t.rho_rect, (int64_t)K * m));
    TRY(tarena.alloc(&t.dinv, (int64_t)K * n)); TRY(tarena.alloc(&t.alpha_in, (int64_t)K * ni));
    TRY(tarena.alloc(&t.grho_all, (int64_t)K * m)); TRY(tarena.alloc(&t.galpha_all, (int64_t)K * ni));
    TRY(tarena.alloc(&t.sigma_dev, K));
    return COSMO_OK;
  }

  // ----------------------------------------------------------- launches --
  cudaEvent_t get_event() {
    if (!ev_pool.empty()) { cudaEvent_t e = ev_pool.back(); ev_pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }

  // CUDA-event timing of a launch (or launch group) of class `tag`; inside a
  // stream capture the events become event-record nodes of the graph
  Rec rec_begin(const char* tag, cudaStream_t st) {
    Rec r{tag, nullptr, nullptr, capturing};
    if (prof_mode != 0 && (prof_mode == 1 || prof_tag == tag)) {
      r.e0 = get_event();
      r.e1 = get_event();
      if (capturing) cudaEventRecordWithFlags(r.e0, st, cudaEventRecordExternal);
      else cudaEventRecord(r.e0, st);
    }
    return r;
  }
  void rec_end(const Rec& r, cudaStream_t st) {
    if (!r.e0) return;
    if (capturing) {
      cudaEventRecordWithFlags(r.e1, st, cudaEventRecordExternal);
      cap_recs.push_back(r);
    } else {
      cudaEventRecord(r.e1, st);
      prof_pending.push_back(r);
    }
  }

  template <class Kern, class... Args>
  void launch(const char* tag, Kern kern, int grid, int block, size_t smem, cudaStream_t st,
              Args... args) {
    const Rec r = rec_begin(tag, st);
    kern<<<grid, block, smem, st>>>(args...);
    ++seq_kernels;
    rec_end(r, st);
  }

  // the same with a thread-block cluster of cs CTAs along x
  template <class Kern, class... Args>
  void launch_cluster(const char* tag, Kern kern, int grid, int block, size_t smem, cudaStream_t st, int cs,
                      Args... args) {
    const Rec r = rec_begin(tag, st);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
    ++seq_kernels;
    rec_end(r, st);
  }

  // CG launch: one CTA or one cluster of cg_cs CTAs per instance
  // one CTA per instance with the vectors in shared memory when they fit
  static constexpr size_t CG_SMEM_MAX = 200 * 1024;
  size_t cg_local = 0;   // bytes of k_pcg_local for the largest CG instance
  size_t cg_smem_bytes() const { return (size_t)h.cg_vec * sizeof(T); }

  // automatic choice: the shared-memory kernel whenever the vectors fit
  // (measured on the 64-instance SOCP batch: 1326 ms per step against 1528
  // with clusters of 2 over global vectors), clusters for larger instances
  //
  // cg_cluster < 0 forces one CTA-per-instance variant: -1 the vectors in
  // shared memory (k_pcg_smem), -2 vectors and matrices in shared memory
  // (k_pcg_local), -3 global-memory vectors (k_pcg); batch creation rejects a
  // forced variant that does not fit.
  int cg_mode = 0;   // the CG kernel chosen by tuning (a cg_cluster value; 0: the shape rule)
  void launch_pcg(const char* tag, cudaStream_t st, const CgArgs<T>& ca) {
#define COSMO_CG_NT(KER, SMB)                                                      \
  {                                                                                \
    if (h.cg_nt == 512) launch(tag, KER<T, V, 512>, P.n_cg, 512, SMB, st, P, ca);  \
    else if (h.cg_nt == 128) launch(tag, KER<T, V, 128>, P.n_cg, 128, SMB, st, P, ca); \
    else launch(tag, KER<T, V, 256>, P.n_cg, 256, SMB, st, P, ca);                 \
  }
    const size_t smb = cg_smem_bytes();
    const int mode = opt.cg_cluster != 0 ? opt.cg_cluster : cg_mode;
    if (mode == -4) {   // one warp per instance
      launch(tag, k_pcg_warp<T, V, 1>, P.n_cg, 32, 0, st, P, ca);
      return;
    }
    if (mode == -1) {
      COSMO_CG_NT(k_pcg_smem, smb);
      return;
    }
    if (mode == -2) {
      COSMO_CG_NT(k_pcg_local, cg_local);
      return;
    }
    if (mode == -3) {
      COSMO_CG_NT(k_pcg, 0);
      return;
    }
    const int cs = mode > 0 ? mode : (smb <= CG_SMEM_MAX ? 1 : h.cg_cs);
    if (cs == 1 && cg_local <= CG_SMEM_MAX) {
      COSMO_CG_NT(k_pcg_local, cg_local);
      return;
    }
    if (cs == 1 && smb <= CG_SMEM_MAX) {
      COSMO_CG_NT(k_pcg_smem, smb);
      return;
    }
    if (cs == 4)
      launch_cluster(tag, k_pcg<T, V, 512, 4>, P.n_cg * 4, 512, 0, st, 4, P, ca);
    else if (cs == 2)
      launch_cluster(tag, k_pcg<T, V, 512, 2>, P.n_cg * 2, 512, 0, st, 2, P, ca);
    else
      COSMO_CG_NT(k_pcg, 0);
#undef COSMO_CG_NT
  }

  // Fork one launch per PSD bucket onto the bucket streams and join them back
  // into st (captured as parallel graph branches).  Timed as one group.
  template <class F>
  void psd_group(const char* tag, cudaStream_t st, F launch_bucket) {
    const Rec r = rec_begin(tag, st);
    if (buckets.size() == 1) {
      launch_bucket(buckets[0], st);
      ++seq_kernels;
    } else {
      cudaEventRecord(ev_fork, st);
      for (auto& bk : buckets) {
        cudaStreamWaitEvent(bk.s, ev_fork, 0);
        launch_bucket(bk, bk.s);
        cudaEventRecord(bk.done, bk.s);
        ++seq_kernels;
      }
      for (auto& bk : buckets) cudaStreamWaitEvent(st, bk.done, 0);
    }
    rec_end(r, st);
  }

  // A change of what is timed drops the recorded graphs: the next forward /
  // backward records them again with (or without) the event nodes.
  cosmo_status profile_enable(const char* tag) override {
    TRY(profile_collect());
    const int mode = !tag ? 1 : (!*tag ? 0 : 2);
    const std::string t = mode == 2 ? std::string(tag) : std::string();
    if (mode != prof_mode || t != prof_tag) drop_graphs();
    prof_mode = mode;
    prof_tag = t;
    return COSMO_OK;
  }
  cosmo_status profile_collect() {
    for (auto& r : prof_pending) {
      CU(cudaEventSynchronize(r.e1));
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, r.e0, r.e1));
      bool found = false;
      for (auto& a : prof_acc)
        if (a.first == r.tag) { a.second.first += ms; a.second.second += 1; found = true; }
      if (!found) prof_acc.push_back(std::make_pair(std::string(r.tag), std::make_pair((double)ms, (int64_t)1)));
      if (!r.graph) {
        ev_pool.push_back(r.e0);
        ev_pool.push_back(r.e1);
      }
    }
    prof_pending.clear();
    return COSMO_OK;
  }
  cosmo_status profile_read(const char* tag, double* ms, int64_t* n, int32_t reset) override {
    TRY(profile_collect());
    *ms = 0.0;
    *n = 0;
    for (auto& a : prof_acc)
      if (!tag || a.first == tag) { *ms += a.second.first; *n += a.second.second; }
    if (reset) prof_acc.clear();
    return COSMO_OK;
  }

  T* st_x(int slot) { return xs + (int64_t)slot * h.n; }
  T* st_s(int slot) { return ss + (int64_t)slot * h.m; }
  T* st_y(int slot) { return ys + (int64_t)slot * h.m; }

  void enqueue_prep(cudaStream_t st) {
    const int64_t Km = (int64_t)K * h.m;
    launch("rho_check", k_rho_copy_check<T, V>, grid_for(Km, 256), 256, 0, st, P, K, (const T*)rho_in, rho_rect, flags);
    if (P.nrect) {
      if (rect_small) launch("rho_rectify", k_rho_rectify<T, V, 8>, grid_for((int64_t)K * P.nrect * 8, 256, INT32_MAX), 256, 0, st, P, K, (const T*)rho_in, rho_rect);
      else launch("rho_rectify", k_rho_rectify<T, V, 32>, grid_for((int64_t)K * P.nrect * 32, 256, INT32_MAX), 256, 0, st, P, K, (const T*)rho_in, rho_rect);
    }
    launch("alpha_check", k_alpha_check<T, V>, grid_for((int64_t)K * h.ninst, 256), 256, 0, st, P, K, (const T*)alpha_in, flags);
    launch("precond", k_precond<T, V>, grid_for((int64_t)K * h.n, 256), 256, 0, st, P, K, (const double*)sigma_dev, (const T*)rho_rect, dinv);
  }

  // one forward step k; state slot `slot` -> slot+1, tape slot `slot`;
  // xt_warm / U_prev: x~ and PSD eigenvectors of step k-1 (null at k = 0)
  void enqueue_step(int32_t k, int slot, const T* xt_warm, const T* U_prev, cudaStream_t st) {
    const T* rho = rho_rect + (int64_t)k * h.m;
    const T* alpha = alpha_in + (int64_t)k * h.ninst;
    const double sig = sigma_h[k];
    T* xt = xts + (int64_t)slot * h.n;
    T* stt = sts + (int64_t)slot * h.m;
    launch("rhs", k_rhs<T, V>, grid_for(h.n, 256), 256, 0, st, P, sig, (const T*)st_x(slot),
           (const T*)st_s(slot), (const T*)st_y(slot), rho, xi,
           (const T*)(dinv + (int64_t)k * h.n), xt);
    CgArgs<T> ca{};
    ca.rhs = xi; ca.x = xt; ca.x0 = xt_warm; ca.rho = rho; ca.dinv = dinv + (int64_t)k * h.n;
    ca.sigma = sig; ca.r = cg_r; ca.p = cg_p; ca.u = cg_u; ca.t = cg_t; ca.tol = opt.cg_tol;
    ca.maxit = opt.cg_max_iter; ca.zero_start = xt_warm ? 0 : 1; ca.flag_bit = F_CG_CAP;
    ca.flags = flags; ca.iters = nullptr; ca.stats = stats + 2;
    if (P.n_cg) launch_pcg("pcg", st, ca);
    StepPtrs<T> sp{};
    sp.x = st_x(slot); sp.s = st_s(slot); sp.y = st_y(slot);
    sp.xn = st_x(slot + 1); sp.sn = st_s(slot + 1); sp.yn = st_y(slot + 1);
    sp.rho = rho; sp.alpha = alpha; sp.xt = xt; sp.st = stt;
    sp.lam = lams + (int64_t)slot * h.sum_p; sp.U = Us + (int64_t)slot * h.sum_p2; sp.flags = flags;
    launch("post", k_post<T, V>, grid_for(h.m + h.n, 256), 256, 0, st, P, sp);
    if (P.nsoc) launch("soc_fwd", k_soc_fwd<T, V>, grid_for((int64_t)P.nsoc * 32, 256, INT32_MAX), 256, 0, st, P, sp);
    if (P.npsd) {
      PsdIterIO<T> io{stt, st_s(slot), st_y(slot), rho, alpha, st_s(slot + 1), st_y(slot + 1), P.row_inst};
      psd_group("psd_fwd", st, [&](const Bucket& bk, cudaStream_t s) {
        psd_fwd_bucket(bk, s, io, sp.lam, sp.U, (opt.eig_warm_start && bk.warm_fits) ? U_prev : nullptr, flags, stats);
      });
    }
  }

  // the forward projection of one PSD class (kernel chosen by the class's method / variant / CTA size)
  void psd_fwd_bucket(const Bucket& bk, cudaStream_t s, const PsdIterIO<T>& io, T* lam, T* U, const T* up,
                      int32_t* fl, unsigned long long* stt) {
    if (bk.method == 2) {
      k_psd_fwd_tpb<T, V, TPB_NT><<<(bk.count + TPB_NT - 1) / TPB_NT, TPB_NT, tpb_smem<T>(TPB_NT), s>>>(
          P, io, lam, U, opt.eig_tol, opt.eig_max_sweeps, fl, bk.start, bk.count, stt, up);
      return;
    }
    if (bk.method == 1) {
      // the working matrix in shared memory when the class's largest block fits
      const int zsm = (int64_t)tql_smem_z<T>(bk.maxp, 256) <= (int64_t)smem_max ? 1 : 0;
      k_psd_fwd_tql<T, V, 256><<<bk.count, 256, zsm ? tql_smem_z<T>(bk.maxp, 256) : tql_smem<T>(bk.maxp, 256), s>>>(
          P, io, lam, U, fl, bk.start, stt, 30 * 4, zsm);
      return;
    }
    if (bk.variant == 3) {
      jt2_for<T>(jt2_pmax(bk.maxp), bk.fnt, [&](auto c, auto pmc, auto ntc) {
        using C = decltype(c);
        constexpr int PM = decltype(pmc)::value, NT_ = decltype(ntc)::value;
        k_psd_fwd_jt2<T, V, NT_, PM, C::TI, C::CI><<<bk.count, NT_, Jt2Geo<T, PM>::bytes(NT_), s>>>(
            P, io, lam, U, opt.eig_tol, opt.eig_max_sweeps, fl, bk.start, stt, up);
      });
      return;
    }
    if (bk.variant == 2) {
      const size_t sm = jt_smem<T>(bk.maxp, bk.fnt);
#define COSMO_JT_LAUNCH(NT_, IPT_) \
  k_psd_fwd_jt<T, V, NT_, IPT_><<<bk.count, NT_, sm, s>>>(P, io, lam, U, opt.eig_tol, opt.eig_max_sweeps, fl, bk.start, stt, up)
#define COSMO_JT_IPT(NT_) \
  { if (bk.tpt == 2) COSMO_JT_LAUNCH(NT_, 2); else if (bk.tpt == 4) COSMO_JT_LAUNCH(NT_, 4); else COSMO_JT_LAUNCH(NT_, 8); }
      if (bk.fnt == 1024) COSMO_JT_IPT(1024)
      else if (bk.fnt == 512) COSMO_JT_IPT(512)
      else if (bk.fnt == 256) COSMO_JT_IPT(256)
      else COSMO_JT_IPT(128)
#undef COSMO_JT_IPT
#undef COSMO_JT_LAUNCH
      return;
    }
    const size_t sm = up ? psd_fwd_smem_warm<T>(bk.maxp, bk.fnt) : psd_fwd_smem<T>(bk.maxp, bk.fnt);
    if (bk.fnt == 512)
      k_psd_fwd<T, V, 512><<<bk.count, 512, sm, s>>>(P, io, lam, U, opt.eig_tol, opt.eig_max_sweeps, fl, bk.start, stt, up);
    else if (bk.fnt == 256)
      k_psd_fwd<T, V, 256><<<bk.count, 256, sm, s>>>(P, io, lam, U, opt.eig_tol, opt.eig_max_sweeps, fl, bk.start, stt, up);
    else
      k_psd_fwd<T, V, 128><<<bk.count, 128, sm, s>>>(P, io, lam, U, opt.eig_tol, opt.eig_max_sweeps, fl, bk.start, stt, up);
  }

  // the Daleckii-Krein backward of one PSD class
  void psd_bwd_bucket(const Bucket& bk, cudaStream_t s, const PsdBwdIO<T>& io, const T* lam, const T* U,
                      int32_t* fl) {
    if (bk.method == 2) {
      k_psd_bwd_tpb<T, V, TPB_NT><<<(bk.count + TPB_NT - 1) / TPB_NT, TPB_NT, tpb_smem<T>(TPB_NT), s>>>(
          P, io, lam, U, opt.dk_gap_tau, bk.start, bk.count);
      return;
    }
    if (bk.method == 1) {
      k_psd_bwd_global<T, V, 256><<<bk.count, 256, 0, s>>>(P, io, lam, U, dk_work, opt.dk_gap_tau, bk.start);
      return;
    }
    if constexpr (std::is_same<T, float>::value) {
      if (opt.dk_tensor_cores && bk.maxp <= DK_TC_MAXP) {
        k_psd_bwd_tc<V><<<bk.count, DK_TC_NT, dk_tc_smem(bk.maxp), s>>>(P, io, lam, U, opt.dk_gap_tau, bk.start, fl);
        return;
      }
    }
    const size_t sm = psd_bwd_smem<T>(bk.maxp, bk.nt);
    if (bk.nt == 512)
      k_psd_bwd<T, V, 512><<<bk.count, 512, sm, s>>>(P, io, lam, U, opt.dk_gap_tau, bk.start);
    else if (bk.nt == 256)
      k_psd_bwd<T, V, 256><<<bk.count, 256, sm, s>>>(P, io, lam, U, opt.dk_gap_tau, bk.start);
    else
      k_psd_bwd<T, V, 128><<<bk.count, 128, sm, s>>>(P, io, lam, U, opt.dk_gap_tau, bk.start);
  }

  // run steps [k0, k1) of segment seg (slot 0 holds z^{k0})
  void enqueue_segment(int32_t seg, cudaStream_t st) {
    const int32_t k0 = seg * cK, k1 = std::min(K, k0 + cK);
    if constexpr (std::is_same<T, float>::value && std::is_same<V, float>::value) {
      if (persist_now()) {
        // one launch per size class for the whole segment (kernels_persist.cuh)
        PersistArgs<T> a{};
        a.k0 = k0; a.k1 = k1;
        a.rho = rho_rect; a.alpha = alpha_in; a.sigma = sigma_dev; a.dinv = dinv;
        a.xs = xs; a.ss = ss; a.ys = ys; a.xts = xts; a.sts = sts; a.lams = lams; a.Us = Us;
        a.U_warm = k0 > 0 ? ck_U + (int64_t)seg * h.sum_p2 : nullptr;
        a.sum_p = h.sum_p; a.sum_p2 = h.sum_p2;
        a.tol = opt.eig_tol; a.max_sweeps = opt.eig_max_sweeps; a.flags = flags; a.stats = stats;
        psd_group("fwd_persist", st, [&](const Bucket& bk, cudaStream_t s) {
          const int warm = (opt.eig_warm_start && bk.warm_fits) ? 1 : 0;
          jt2_for<T>(jt2_pmax(bk.maxp), bk.fnt, [&](auto c, auto pmc, auto ntc) {
            using C = decltype(c);
            constexpr int PM = decltype(pmc)::value, NT_ = decltype(ntc)::value;
            k_fwd_persist_jt2<T, V, NT_, PM, C::TI, C::CI><<<bk.count, NT_, Jt2Geo<T, PM>::bytes(NT_), s>>>(
                P, a, bk.start, warm);
          });
        });
        return;
      }
    }
    for (int32_t k = k0; k < k1; ++k) {
      const int slot = k - k0;
      const T* warm = nullptr;
      const T* uprev = nullptr;
      if (k > 0) {
        warm = slot == 0 ? ck_xt + (int64_t)seg * h.n : xts + (int64_t)(slot - 1) * h.n;
        uprev = slot == 0 ? ck_U + (int64_t)seg * h.sum_p2 : Us + (int64_t)(slot - 1) * h.sum_p2;
      }
      enqueue_step(k, slot, warm, uprev, st);
      if (lr_track) enqueue_norms(slot + 1, k + 1, st);
      // xi^{k+1} from z^{k+1}, s^k and s~^{k+1} gives the parameters of step k + 2
      if (pol_mode && k + 1 <= K - 2) enqueue_pol(k + 1, slot + 1, st_s(slot), sts + (int64_t)slot * h.m, st);
    }
  }

  // ||r_p||^2, ||r_d||^2 of the state in `slot` into the log-ratio buffers at step index k
  void enqueue_norms(int slot, int32_t k, cudaStream_t st) {
    ResArgs<T> ra{st_x(slot), st_s(slot), st_y(slot), nullptr, nullptr,
                  lr_rp2 + (int64_t)k * h.ninst, lr_rd2 + (int64_t)k * h.ninst, nullptr, nullptr};
    launch("residuals", k_residuals<T, V, 256>, h.ninst, 256, 0, st, P, ra);
  }

  void copy_state(T* dx, T* ds, T* dy, const T* sx, const T* s_, const T* sy, cudaStream_t st) {
    cudaMemcpyAsync(dx, sx, sizeof(T) * h.n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(ds, s_, sizeof(T) * h.m, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(dy, sy, sizeof(T) * h.m, cudaMemcpyDeviceToDevice, st);
  }

  int32_t last_len() const { return K - (nseg - 1) * cK; }

  // whole forward: prep, all segments with checkpoints, optional loss
  void enqueue_forward(bool want_loss, cudaStream_t st) {
    if (pol_mode) enqueue_pol_prep(st);
    else enqueue_prep(st);
    lr_track = want_loss && opt.loss_kind == 1;
    if (lr_track) enqueue_norms(0, 0, st);
    for (int32_t seg = 0; seg < nseg; ++seg) {
      if (seg > 0) {
        // slot cK of the previous segment is z^{seg*cK}; x~ of its last step warms CG
        copy_state(st_x(0), st_s(0), st_y(0), st_x(cK), st_s(cK), st_y(cK), st);
        cudaMemcpyAsync(ck_xt + (int64_t)seg * h.n, xts + (int64_t)(cK - 1) * h.n,
                        sizeof(T) * h.n, cudaMemcpyDeviceToDevice, st);
        if (h.sum_p2)
          cudaMemcpyAsync(ck_U + (int64_t)seg * h.sum_p2, Us + (int64_t)(cK - 1) * h.sum_p2,
                          sizeof(T) * h.sum_p2, cudaMemcpyDeviceToDevice, st);
      }
      copy_state(ck_x + (int64_t)seg * h.n, ck_s + (int64_t)seg * h.m, ck_y + (int64_t)seg * h.m,
                 st_x(0), st_s(0), st_y(0), st);
      enqueue_segment(seg, st);
    }
    lr_track = false;
    if (want_loss && opt.loss_kind == 1) {
      launch("residuals", k_logratio_loss, (h.ninst + 127) / 128, 128, 0, st, h.ninst, K, (const double*)lr_rd2,
             (const double*)lr_rp2, loss_buf);
    } else if (want_loss) {
      const int fs = last_len();
      ResArgs<T> ra{st_x(fs), st_s(fs), st_y(fs), rp, rd, nullptr, nullptr, nullptr, loss_buf};
      launch("residuals", k_residuals<T, V, 256>, h.ninst, 256, 0, st, P, ra);
    }
  }

  void enqueue_bwd_step(int32_t k, int slot, int cur, cudaStream_t st) {
    BwdPtrs<T> q{};
    q.x = st_x(slot); q.s = st_s(slot); q.y = st_y(slot); q.sn = st_s(slot + 1);
    q.rho = rho_rect + (int64_t)k * h.m; q.alpha = alpha_in + (int64_t)k * h.ninst;
    q.sigma = sigma_h[k];
    q.xt = xts + (int64_t)slot * h.n; q.st = sts + (int64_t)slot * h.m;
    q.lam = lams + (int64_t)slot * h.sum_p; q.U = Us + (int64_t)slot * h.sum_p2;
    q.xb = xb[cur]; q.sb = sb[cur]; q.yb = yb[cur];
    q.xb2 = xb[cur ^ 1]; q.sb2 = sb[cur ^ 1]; q.yb2 = yb[cur ^ 1];
    q.gproj = gproj; q.vbar = vbar; q.adjrhs = adjrhs; q.lamt = lamt;
    q.grho = grho_all + (int64_t)k * h.m; q.galpha = galpha_all + (int64_t)k * h.ninst;
    q.flags = flags; q.dk_tau = opt.dk_gap_tau; q.dinv = dinv + (int64_t)k * h.n;
    launch("bwd_gproj", k_bwd_gproj<T, V>, grid_for(h.m, 256), 256, 0, st, P, q);
    if (P.nsoc) launch("soc_bwd", k_soc_bwd<T, V>, grid_for((int64_t)P.nsoc * 32, 256, INT32_MAX), 256, 0, st, P, q);
    if (P.npsd) {
      PsdBwdIO<T> io{gproj, vbar, P.row_inst};
      psd_group("psd_bwd", st, [&](const Bucket& bk, cudaStream_t s) { psd_bwd_bucket(bk, s, io, q.lam, q.U, flags); });
    }
    launch("bwd_relax", k_bwd_relax<T, V, 512>, h.ninst, 512, 0, st, P, q);
    CgArgs<T> ca{};
    ca.rhs = adjrhs; ca.x = lamt; ca.x0 = nullptr; ca.rho = q.rho;
    ca.dinv = dinv + (int64_t)k * h.n; ca.sigma = q.sigma; ca.r = cg_r; ca.p = cg_p; ca.u = cg_u;
    ca.t = cg_t; ca.tol = opt.cg_tol; ca.maxit = opt.cg_max_iter; ca.zero_start = 1;
    ca.flag_bit = F_ADJ_CG_CAP; ca.flags = flags; ca.iters = nullptr; ca.stats = stats + 4;
    if (P.n_cg) launch_pcg("pcg_adj", st, ca);
    launch("bwd_solve", k_bwd_solve<T, V>, grid_for(h.m + h.n, 256), 256, 0, st, P, q);
  }

  // whole backward (cotangents staged in gx_in/gs_in/gy_in/gloss_buf)
  void enqueue_backward(bool use_gloss, cudaStream_t st) {
    const int fs = last_len();
    const bool logratio = opt.loss_kind == 1;
    // log-ratio loss: the seed carries only the caller's cotangents; every
    // state's loss term is injected on the way back
    SeedArgs<T> sa{rp, rd, (use_gloss && !logratio) ? gloss_buf : nullptr, gx_in, gs_in, gy_in,
                   xb[0], sb[0], yb[0]};
    (void)fs;
    launch("loss_seed", k_loss_seed<T, V>, grid_for(h.m + h.n, 256), 256, 0, st, P, sa);
    int cur = 0;
    for (int32_t seg = nseg - 1; seg >= 0; --seg) {
      if (seg != nseg - 1) {
        copy_state(st_x(0), st_s(0), st_y(0), ck_x + (int64_t)seg * h.n, ck_s + (int64_t)seg * h.m,
                   ck_y + (int64_t)seg * h.m, st);
        enqueue_segment(seg, st);
      }
      const int32_t k0 = seg * cK, k1 = std::min(K, k0 + cK);
      for (int32_t k = k1 - 1; k >= k0; --k) {
        if (logratio && use_gloss) {
          // cotangent of state k + 1's term, added to the one step k receives
          const int sl = k + 1 - k0;
          ResArgs<T> ra{st_x(sl), st_s(sl), st_y(sl), rp, rd, nullptr, nullptr, nullptr, nullptr};
          launch("residuals", k_residuals<T, V, 256>, h.ninst, 256, 0, st, P, ra);
          launch("loss_seed", k_logratio_w<T>, (h.ninst + 127) / 128, 128, 0, st, h.ninst, k + 1,
                 (const double*)lr_rd2, (const double*)lr_rp2, (const double*)gloss_buf, lr_wa, lr_wb);
          launch("loss_seed", k_logratio_seed<T, V>, grid_for(h.m + h.n, 256), 256, 0, st, P, (const T*)rp,
                 (const T*)rd, (const T*)lr_wa, (const T*)lr_wb, xb[cur], sb[cur], yb[cur]);
        }
        enqueue_bwd_step(k, k - k0, cur, st);
        cur ^= 1;
      }
    }
    if (P.nrect) {
      if (rect_small) launch("rect_adjoint", k_rect_adjoint<T, V, 8>, grid_for((int64_t)K * P.nrect * 8, 256, INT32_MAX), 256, 0, st, P, K, grho_all);
      else launch("rect_adjoint", k_rect_adjoint<T, V, 32>, grid_for((int64_t)K * P.nrect * 32, 256, INT32_MAX), 256, 0, st, P, K, grho_all);
    }
    final_cot = cur;
  }
  int final_cot = 0;

  // run `fn` either captured into a cached graph or directly on st
  // graph recs: release (after collecting what is pending) when the graph goes
  cosmo_status release_recs(std::vector<Rec>& recs) {
    if (recs.empty()) return COSMO_OK;
    TRY(profile_collect());
    for (auto& r : recs) { ev_pool.push_back(r.e0); ev_pool.push_back(r.e1); }
    recs.clear();
    return COSMO_OK;
  }
  template <class Fn>
  cosmo_status run_seq(cudaGraphExec_t& exec, int64_t& nk, std::vector<Rec>& recs, bool reuse, Fn fn,
                       cudaStream_t st) {
    if (!opt.use_graph) {
      seq_kernels = 0;
      fn(st);
      CU(cudaGetLastError());
      launched += seq_kernels;
      g_launches += seq_kernels;
      return COSMO_OK;
    }
    if (!(exec && reuse)) {
      if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
      TRY(release_recs(recs));
      seq_kernels = 0;
      cap_recs.clear();
      CU(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      capturing = true;
      fn(cap);
      capturing = false;
      recs = cap_recs;
      cap_recs.clear();
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(cap, &g);
      if (e != cudaSuccess) return fail(COSMO_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { exec = nullptr; return fail(COSMO_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e)); }
      nk = seq_kernels;
    }
    if (!recs.empty()) {
      // the previous replay's events are read before they are recorded again
      TRY(profile_collect());
      for (auto& r : recs) prof_pending.push_back(r);
    }
    CU(cudaGraphLaunch(exec, st));
    launched += nk;
    g_launches += nk;
    return COSMO_OK;
  }

  cosmo_status forward(int32_t K_, const double* sigma, const void* rho, const void* alpha,
                       const void* x0, const void* s0, const void* y0, void* xK, void* sK,
                       void* yK, double* loss, int32_t tape, cudaStream_t st) override {
    if (K_ < 1) return fail(COSMO_E_INVAL, "K must be >= 1");
    if (!pol_mode && (!rho || !alpha)) return fail(COSMO_E_INVAL, "rho and alpha are required");
    TRY(ensure_tape(K_));
    std::vector<double> sg(K, 1e-6);
    if (sigma)
      for (int32_t k = 0; k < K; ++k) {
        if (!(sigma[k] > 0.0) || !std::isfinite(sigma[k])) return fail(COSMO_E_INVAL, "sigma must be > 0");
        sg[k] = sigma[k];
      }
    sigma_h = sg;
    const int64_t n = h.n, m = h.m;
    CU(cudaMemcpyAsync(sigma_dev, sg.data(), sizeof(double) * K, cudaMemcpyHostToDevice, st));
    if (!pol_mode) {
      CU(cudaMemcpyAsync(rho_in, rho, sizeof(T) * K * m, cudaMemcpyDeviceToDevice, st));
      CU(cudaMemcpyAsync(alpha_in, alpha, sizeof(T) * K * h.ninst, cudaMemcpyDeviceToDevice, st));
    }
    pol_valid = false;
    if (x0) CU(cudaMemcpyAsync(st_x(0), x0, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
    else CU(cudaMemsetAsync(st_x(0), 0, sizeof(T) * n, st));
    if (s0) CU(cudaMemcpyAsync(st_s(0), s0, sizeof(T) * m, cudaMemcpyDeviceToDevice, st));
    else CU(cudaMemsetAsync(st_s(0), 0, sizeof(T) * m, st));
    if (y0) CU(cudaMemcpyAsync(st_y(0), y0, sizeof(T) * m, cudaMemcpyDeviceToDevice, st));
    else CU(cudaMemsetAsync(st_y(0), 0, sizeof(T) * m, st));
    const bool want_loss = loss != nullptr || tape;
    const bool reuse = gfwd_key[0] == K && gfwd_key[1] == (int)want_loss && gfwd_key[2] == (int)pol_mode &&
                       gfwd_sigma == sg;
    TRY(run_seq(gfwd, gfwd_nk, gfwd_recs, reuse, [&](cudaStream_t s) { enqueue_forward(want_loss, s); }, st));
    gfwd_key[0] = K; gfwd_key[1] = (int)want_loss; gfwd_key[2] = (int)pol_mode; gfwd_sigma = sg;
    seg_in_buffer = nseg - 1;
    tape_valid = tape != 0;
    loss_valid = want_loss;
    const int fs = last_len();
    if (xK) CU(cudaMemcpyAsync(xK, st_x(fs), sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
    if (sK) CU(cudaMemcpyAsync(sK, st_s(fs), sizeof(T) * m, cudaMemcpyDeviceToDevice, st));
    if (yK) CU(cudaMemcpyAsync(yK, st_y(fs), sizeof(T) * m, cudaMemcpyDeviceToDevice, st));
    if (loss) CU(cudaMemcpyAsync(loss, loss_buf, sizeof(double) * h.ninst, cudaMemcpyDeviceToDevice, st));
    return COSMO_OK;
  }

  cosmo_status backward(const void* gx, const void* gs, const void* gy, const double* gl,
                        void* grho, void* galpha, void* gx0, void* gs0, void* gy0,
                        cudaStream_t st) override {
    if (!tape_valid) return fail(COSMO_E_STATE, "backward needs a forward with record_tape=1");
    const int64_t n = h.n, m = h.m;
    // the last segment must be in the buffer (a previous backward may have replaced it)
    if (seg_in_buffer != nseg - 1) {
      const int32_t seg = nseg - 1;
      seq_kernels = 0;
      copy_state(st_x(0), st_s(0), st_y(0), ck_x + (int64_t)seg * n, ck_s + (int64_t)seg * m,
                 ck_y + (int64_t)seg * m, st);
      enqueue_segment(seg, st);
      CU(cudaGetLastError());
      launched += seq_kernels;
      g_launches += seq_kernels;
      seg_in_buffer = seg;
    }
    if (gx) CU(cudaMemcpyAsync(gx_in, gx, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
    else CU(cudaMemsetAsync(gx_in, 0, sizeof(T) * n, st));
    if (gs) CU(cudaMemcpyAsync(gs_in, gs, sizeof(T) * m, cudaMemcpyDeviceToDevice, st));
    else CU(cudaMemsetAsync(gs_in, 0, sizeof(T) * m, st));
    if (gy) CU(cudaMemcpyAsync(gy_in, gy, sizeof(T) * m, cudaMemcpyDeviceToDevice, st));
    else CU(cudaMemsetAsync(gy_in, 0, sizeof(T) * m, st));
    if (gl) {
      if (!loss_valid) return fail(COSMO_E_STATE, "gloss given but the forward computed no loss");
      CU(cudaMemcpyAsync(gloss_buf, gl, sizeof(double) * h.ninst, cudaMemcpyDeviceToDevice, st));
    } else {
      CU(cudaMemsetAsync(gloss_buf, 0, sizeof(double) * h.ninst, st));
    }
    // rp / rd must exist for the seed kernel even without a loss cotangent
    if (!loss_valid) {
      CU(cudaMemsetAsync(rp, 0, sizeof(T) * m, st));
      CU(cudaMemsetAsync(rd, 0, sizeof(T) * n, st));
    }
    const bool reuse = gbwd_sigma == sigma_h && gbwd != nullptr;
    TRY(run_seq(gbwd, gbwd_nk, gbwd_recs, reuse, [&](cudaStream_t s) { enqueue_backward(true, s); }, st));
    gbwd_sigma = sigma_h;
    seg_in_buffer = nseg > 1 ? 0 : nseg - 1;
    const int c = final_cot;  // each reverse step swaps the cotangent buffers
    if (grho) CU(cudaMemcpyAsync(grho, grho_all, sizeof(T) * K * m, cudaMemcpyDeviceToDevice, st));
    if (galpha) CU(cudaMemcpyAsync(galpha, galpha_all, sizeof(T) * K * h.ninst, cudaMemcpyDeviceToDevice, st));
    if (gx0) CU(cudaMemcpyAsync(gx0, xb[c], sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
    if (gs0) CU(cudaMemcpyAsync(gs0, sb[c], sizeof(T) * m, cudaMemcpyDeviceToDevice, st));
    if (gy0) CU(cudaMemcpyAsync(gy0, yb[c], sizeof(T) * m, cudaMemcpyDeviceToDevice, st));
    return COSMO_OK;
  }

  // ---- solve to tolerance (vanilla COSMO with residual balancing) ----
  DevArena sarena;                      // solve buffers, sized for sv_c steps per chunk
  int32_t sv_c = 0;
  T *sv_rho = nullptr, *sv_alpha = nullptr;
  double *sv_rhoi = nullptr, *sv_nrm = nullptr, *sv_rbp = nullptr, *sv_rbd = nullptr;
  int32_t *sv_conv = nullptr, *sv_run = nullptr, *sv_run_h = nullptr;

  cosmo_status solve(const cosmo_solve_params& p, void* x, void* s, void* y, int32_t* iters, double* rbp,
                     double* rbd, double* rho, cudaStream_t st) override {
    const int c = p.check_every;
    if (!x || !s || !y || !(p.sigma > 0.0) || !(p.alpha > 0.0 && p.alpha < 2.0) || !(p.rho0 > 0.0) ||
        !(p.rho_eq_scale > 0.0) || !(p.eps > 0.0) || !(p.rebalance_tol >= 1.0) || !(p.rho_min > 0.0) ||
        !(p.rho_max >= p.rho_min) || p.max_iter < 1 || c < 1 || p.rebalance_every < 0 ||
        (p.rebalance_every > 0 && p.rebalance_every % c != 0))
      return fail(COSMO_E_INVAL, "bad arguments to cosmo_solve");
    const int64_t m = h.m;
    const int32_t ni = h.ninst;
    if (sv_c != c) {
      if (sv_run_h) { cudaFreeHost(sv_run_h); sv_run_h = nullptr; }
      sarena.release();
      TRY(sarena.alloc(&sv_rho, (int64_t)c * std::max<int64_t>(m, 1)));
      TRY(sarena.alloc(&sv_alpha, (int64_t)c * ni));
      TRY(sarena.alloc(&sv_rhoi, ni)); TRY(sarena.alloc(&sv_nrm, 8 * (int64_t)ni));
      TRY(sarena.alloc(&sv_rbp, ni)); TRY(sarena.alloc(&sv_rbd, ni));
      TRY(sarena.alloc(&sv_conv, ni)); TRY(sarena.alloc(&sv_run, 1));
      CU(cudaMallocHost(&sv_run_h, sizeof(int32_t)));
      sv_c = c;
    }
    std::vector<double> r0(ni, p.rho0);
    CU(cudaMemcpyAsync(sv_rhoi, r0.data(), sizeof(double) * ni, cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(sv_conv, 0xff, sizeof(int32_t) * ni, st));   // -1: not yet converged
    std::vector<double> sig(c, p.sigma);
    int32_t it = 0;
    while (it < p.max_iter) {
      const int32_t kk = std::min(c, p.max_iter - it);
      k_solve_fill<T, V><<<grid_for((int64_t)kk * std::max<int64_t>(m, ni), 256), 256, 0, st>>>(
          P, kk, sv_rhoi, p.rho_eq_scale, p.alpha, sv_rho, sv_alpha);
      TRY(forward(kk, sig.data(), sv_rho, sv_alpha, x, s, y, x, s, y, nullptr, 0, st));
      it += kk;
      k_kkt_inf<T, V, 256><<<ni, 256, 0, st>>>(P, (const T*)x, (const T*)s, (const T*)y, sv_nrm);
      CU(cudaMemsetAsync(sv_run, 0, sizeof(int32_t), st));
      SolveCtl ctl{p.eps, p.rebalance_tol, p.rho_min, p.rho_max, it,
                   p.rebalance_every > 0 && it % p.rebalance_every == 0 ? 1 : 0};
      k_solve_update<<<(ni + 127) / 128, 128, 0, st>>>(ni, sv_nrm, ctl, sv_rhoi, sv_conv, sv_rbp, sv_rbd, sv_run);
      CU(cudaGetLastError());
      launched += 3; g_launches += 3;
      CU(cudaMemcpyAsync(sv_run_h, sv_run, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      if (*sv_run_h == 0) break;
    }
    if (iters) CU(cudaMemcpyAsync(iters, sv_conv, sizeof(int32_t) * ni, cudaMemcpyDeviceToHost, st));
    if (rbp) CU(cudaMemcpyAsync(rbp, sv_rbp, sizeof(double) * ni, cudaMemcpyDeviceToHost, st));
    if (rbd) CU(cudaMemcpyAsync(rbd, sv_rbd, sizeof(double) * ni, cudaMemcpyDeviceToHost, st));
    if (rho) CU(cudaMemcpyAsync(rho, sv_rhoi, sizeof(double) * ni, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return COSMO_OK;
  }

  // ---- warm-start network (App. E) ----
  DevArena warena;   // features and reverse-pass buffers, allocated on first use
  T *ws_ctx = nullptr, *ws_fx = nullptr, *ws_fc = nullptr, *ws_g = nullptr;
  T *ws_h1 = nullptr, *ws_d1 = nullptr, *ws_h2 = nullptr, *ws_d2 = nullptr;
  double* ws_part = nullptr;
  bool ws_feat_ok = false, ws_bwd_ok = false;

  // ctx and the feature matrices, recomputed on every call (q and b are read
  // from the batch as they stand)
  cosmo_status ws_features(cudaStream_t st) {
    if (!ws_feat_ok) {
      TRY(warena.alloc(&ws_ctx, 4 * (int64_t)h.ninst));
      TRY(warena.alloc(&ws_fx, (int64_t)WS_NFX * h.n));
      TRY(warena.alloc(&ws_fc, (int64_t)WS_NFC * h.m));
      ws_feat_ok = true;
    }
    launch("ws_feat", k_ws_ctx<T, V, 256>, h.ninst, 256, 0, st, P, ws_ctx);
    if (h.n + h.m > 0) launch("ws_feat", k_ws_feat<T, V>, grid_for(h.n + h.m, 256), 256, 0, st, P, (const T*)ws_ctx,
                              ws_fx, ws_fc);
    CU(cudaGetLastError());
    launched += 2; g_launches += 2;
    return COSMO_OK;
  }

  cosmo_status ws_forward(const void* tx, const void* tc, void* x0, void* s0, void* y0,
                          cudaStream_t st) override {
    if (!tx || !tc || !x0 || (h.m > 0 && (!s0 || !y0)))
      return fail(COSMO_E_INVAL, "bad arguments to cosmo_ws_forward");
    TRY(ws_features(st));
    if (h.n > 0)
      launch("ws_fwd", k_ws_fwd<T, WS_NFX, 1>, (int)((h.n + 127) / 128), 128, sizeof(T) * ws_nparams(WS_NFX, 1), st,
             h.n, (const T*)ws_fx, (const T*)tx, (T*)x0, (T*)nullptr);
    if (h.m > 0)
      launch("ws_fwd", k_ws_fwd<T, WS_NFC, 2>, (int)((h.m + 127) / 128), 128, sizeof(T) * ws_nparams(WS_NFC, 2), st,
             h.m, (const T*)ws_fc, (const T*)tc, (T*)s0, (T*)y0);
    CU(cudaGetLastError());
    launched += 2; g_launches += 2;
    return COSMO_OK;
  }

  // the weight-sum kernel with the thread shape fitted to the (KA + 1) x KB output
  void atb(int nch, int64_t chunk, int64_t N, const T* A, int64_t lda, int KA, const T* B, int64_t ldb, int KB,
           double* part, cudaStream_t st) {
    const int ka = KA + 1;
    if (KB <= 2) {   // output-layer blocks: a streaming column sum
      launch("ws_grad", k_ws_atb_thin<T>, nch, 256, 0, st, N, chunk, A, lda, KA, 1, B, ldb, KB, part);
      return;
    }
    if constexpr (std::is_same<T, float>::value) {
      // FP32 blocks 17..64 columns wide: split-TF32 products on the tensor
      // cores (chunk is a multiple of 32).  Measured: the warm start's 9x64
      // and 65x64 blocks 3.3 -> 2.6 ms per step; the policy's 32-wide ones
      // 13.8 -> 12.9 ms once the staging was bank-conflict free; the 65x2
      // and 33x1 output-layer blocks stay on the CUDA cores.
      if (opt.dk_tensor_cores && KB > 16) {
        if (KB > 32)
          launch("ws_grad", k_ws_atb_tc<64>, nch, 256, ws_tc_smem(64), st, N, chunk, A, lda, KA, 1, B, ldb, KB, part,
                 flags);
        else
          launch("ws_grad", k_ws_atb_tc<32>, nch, 256, ws_tc_smem(32), st, N, chunk, A, lda, KA, 1, B, ldb, KB, part,
                 flags);
        return;
      }
    }
#define COSMO_ATB(RI, RJ, TY, TX) \
  launch("ws_grad", k_ws_atb<T, RI, RJ, TY, TX>, nch, 256, 0, st, N, chunk, A, lda, KA, 1, B, ldb, KB, part)
    if (KB <= 2) {
      if (ka <= 48) COSMO_ATB(3, 1, 16, 2);
      else COSMO_ATB(5, 1, 16, 2);
    } else if (KB <= 32) {
      if (ka <= 8) COSMO_ATB(1, 2, 8, 16);
      else if (ka <= 16) COSMO_ATB(1, 2, 16, 16);
      else if (ka <= 48) COSMO_ATB(3, 2, 16, 16);
      else COSMO_ATB(5, 2, 16, 16);
    } else {
      if (ka <= 16) COSMO_ATB(1, 4, 16, 16);
      else COSMO_ATB(5, 4, 16, 16);
    }
#undef COSMO_ATB
  }

  // gtheta (+)= the parameter gradient of an MLP (F inputs, H x H hidden,
  // O outputs) over elements e < N with features X[f * ldx + e] and output
  // cotangent G[o * ldg + e]; h1..d2 hold H x N reals, part the chunk partials
  template <int F, int O, int H>
  cosmo_status mlp_bwd(int64_t N, const T* X, int64_t ldx, const T* theta, const T* G, int64_t ldg, T* gtheta,
                       int acc, T* h1, T* d1, T* h2, T* d2, double* part, const char* tag, cudaStream_t st) {
    if (N == 0) {
      if (!acc) CU(cudaMemsetAsync(gtheta, 0, sizeof(T) * ws_nparams(F, O, H), st));
      return COSMO_OK;
    }
    launch(tag, k_ws_bwd<T, F, O, H>, (int)((N + 127) / 128), 128, sizeof(T) * ws_nparams(F, O, H), st, N, ldx, X,
           theta, G, ldg, h1, d1, h2, d2);
    // elements per CTA: a multiple of 32 giving at most WS_MAXCH CTAs
    const int64_t chunk = ((N + WS_MAXCH - 1) / WS_MAXCH + WS_TILE - 1) / WS_TILE * WS_TILE;
    const int nch = (int)((N + chunk - 1) / chunk);
    // [W1; b1] = [X; 1] D1', [W2; b2] = [H1; 1] D2', [W3; b3] = [H2; 1] G'
    const T* As[3] = {X, h1, h2};
    const T* Bs[3] = {d1, d2, G};
    const int64_t lda[3] = {ldx, N, N}, ldb[3] = {N, N, ldg};
    const int KA[3] = {F, H, H}, KB[3] = {H, H, O};
    int64_t off = 0;
    for (int l = 0; l < 3; ++l) {
      const int np = (KA[l] + 1) * KB[l];
      atb(nch, chunk, N, As[l], lda[l], KA[l], Bs[l], ldb[l], KB[l], part, st);
      launch("ws_grad", k_ws_sum<T>, (np + 31) / 32, 256, 0, st, nch, np, (const double*)part, gtheta + off, acc);
      off += np;
    }
    CU(cudaGetLastError());
    launched += 7; g_launches += 7;
    return COSMO_OK;
  }

  template <int F, int O>
  cosmo_status ws_mlp_backward(int64_t N, const T* X, const T* theta, const T* G, T* gtheta, cudaStream_t st) {
    return mlp_bwd<F, O, WS_H>(N, X, N, theta, G, N, gtheta, 0, ws_h1, ws_d1, ws_h2, ws_d2, ws_part, "ws_bwd", st);
  }

  cosmo_status ws_backward(const void* tx, const void* tc, const void* gx0, const void* gs0, const void* gy0,
                           void* gtx, void* gtc, cudaStream_t st) override {
    if (!tx || !tc || !gx0 || !gtx || !gtc || (h.m > 0 && (!gs0 || !gy0)))
      return fail(COSMO_E_INVAL, "bad arguments to cosmo_ws_backward");
    if (!ws_bwd_ok) {
      const int64_t nmax = std::max<int64_t>(std::max(h.n, h.m), 1);
      TRY(warena.alloc(&ws_g, 2 * std::max<int64_t>(h.m, 1)));
      TRY(warena.alloc(&ws_h1, WS_H * nmax)); TRY(warena.alloc(&ws_d1, WS_H * nmax));
      TRY(warena.alloc(&ws_h2, WS_H * nmax)); TRY(warena.alloc(&ws_d2, WS_H * nmax));
      TRY(warena.alloc(&ws_part, (int64_t)WS_MAXCH * (WS_H + 1) * WS_H));
      ws_bwd_ok = true;
    }
    TRY(ws_features(st));
    TRY((ws_mlp_backward<WS_NFX, 1>(h.n, ws_fx, (const T*)tx, (const T*)gx0, (T*)gtx, st)));
    if (h.m > 0) {
      CU(cudaMemcpyAsync(ws_g, gs0, sizeof(T) * h.m, cudaMemcpyDeviceToDevice, st));
      CU(cudaMemcpyAsync(ws_g + h.m, gy0, sizeof(T) * h.m, cudaMemcpyDeviceToDevice, st));
    }
    TRY((ws_mlp_backward<WS_NFC, 2>(h.m, ws_fc, (const T*)tc, ws_g, (T*)gtc, st)));
    return COSMO_OK;
  }

  // ---- closed-loop hyperparameter policy (App. E) ----
  DevArena parena;   // sized for pol_K steps
  int32_t pol_K = 0;
  bool pol_mode = false, pol_valid = false;
  int64_t pol_ch = 0;   // elements per chunk of the MLP reverse pass
  T *pol_tr = nullptr, *pol_ta = nullptr, *pol_l0 = nullptr;
  T *pol_Xr = nullptr, *pol_Jr = nullptr, *pol_Gr = nullptr, *pol_lr = nullptr, *pol_glr = nullptr;
  T *pol_Xa = nullptr, *pol_Ja = nullptr, *pol_Ga = nullptr, *pol_la = nullptr, *pol_gla = nullptr;
  T *pol_sc = nullptr, *pol_h1 = nullptr, *pol_d1 = nullptr, *pol_h2 = nullptr, *pol_d2 = nullptr;
  double* pol_part = nullptr;

  cosmo_status pol_alloc(int32_t K_) {
    if (pol_K == K_) return COSMO_OK;
    parena.release();
    pol_K = 0;
    const int64_t m = h.m, ni = h.ninst, Nr = (int64_t)(K_ - 1) * m, Na = (int64_t)(K_ - 1) * ni;
    TRY(parena.alloc(&pol_tr, ws_nparams(POL_NFR, 1, POL_H)));
    TRY(parena.alloc(&pol_ta, ws_nparams(POL_NFA, 1, POL_H)));
    TRY(parena.alloc(&pol_l0, 5));
    TRY(parena.alloc(&pol_Xr, POL_NFR * Nr)); TRY(parena.alloc(&pol_Jr, Nr)); TRY(parena.alloc(&pol_Gr, Nr));
    TRY(parena.alloc(&pol_lr, (int64_t)K_ * m)); TRY(parena.alloc(&pol_glr, m));
    TRY(parena.alloc(&pol_Xa, POL_NFA * Na)); TRY(parena.alloc(&pol_Ja, Na)); TRY(parena.alloc(&pol_Ga, Na));
    TRY(parena.alloc(&pol_la, (int64_t)K_ * ni)); TRY(parena.alloc(&pol_gla, ni));
    TRY(parena.alloc(&pol_sc, 2 * ni));
    pol_ch = std::max<int64_t>(std::min<int64_t>(std::max(Nr, Na), (int64_t)1 << 21), 1);
    TRY(parena.alloc(&pol_h1, POL_H * pol_ch)); TRY(parena.alloc(&pol_d1, POL_H * pol_ch));
    TRY(parena.alloc(&pol_h2, POL_H * pol_ch)); TRY(parena.alloc(&pol_d2, POL_H * pol_ch));
    TRY(parena.alloc(&pol_part, (int64_t)WS_MAXCH * (POL_H + 1) * POL_H));
    pol_K = K_;
    return COSMO_OK;
  }

  // rho_rect and dinv of step k from rho_in[k] (the policy's rho is positive
  // and finite by construction)
  void enqueue_step_params(int32_t k, cudaStream_t st) {
    const int64_t om = (int64_t)k * h.m;
    launch("rho_check", k_rho_copy_check<T, V>, grid_for(h.m, 256), 256, 0, st, P, 1, (const T*)(rho_in + om),
           rho_rect + om, flags);
    if (P.nrect)
      launch("rho_rectify", k_rho_rectify<T, V, 32>, grid_for((int64_t)P.nrect * 32, 256, INT32_MAX), 256, 0, st, P, 1,
             (const T*)(rho_in + om), rho_rect + om);
    launch("precond", k_precond<T, V>, grid_for(h.n, 256), 256, 0, st, P, 1, (const double*)(sigma_dev + k),
           (const T*)(rho_rect + om), dinv + (int64_t)k * h.n);
  }

  // l^0, the parameters of step 0, and xi^0 -> parameters of step 1
  void enqueue_pol_prep(cudaStream_t st) {
    launch("pol_fwd", k_pol_init<T, V>, grid_for(std::max<int64_t>(h.m, h.ninst), 256), 256, 0, st, P,
           (const T*)pol_l0, pol_lr, rho_in, pol_la, alpha_in);
    enqueue_step_params(0, st);
    if (K >= 2) enqueue_pol(0, 0, nullptr, nullptr, st);
  }

  // xi^j of the state in `slot` (s^{j-1} = sprev, s~^j = stil; null at j = 0)
  // -> l^{j+1}, the parameters of step j + 1
  void enqueue_pol(int32_t j, int slot, const T* sprev, const T* stil, cudaStream_t st) {
    const int64_t m = h.m, ni = h.ninst, Nr = (int64_t)(K - 1) * m, Na = (int64_t)(K - 1) * ni;
    launch("pol_fwd", k_pol_inst<T, V, 256>, (int)ni, 256, 0, st, P, (const T*)st_x(slot), (const T*)st_s(slot),
           (const T*)st_y(slot), sprev, stil, (const T*)pol_ta, (const T*)(pol_la + j * ni), pol_la + (j + 1) * ni,
           alpha_in + (j + 1) * ni, pol_Xa + j * ni, Na, pol_Ja + j * ni, pol_sc);
    if (m > 0)
      launch("pol_fwd", k_pol_rows<T, V>, (int)((m + 127) / 128), 128, sizeof(T) * ws_nparams(POL_NFR, 1, POL_H), st,
             P, (const T*)st_x(slot), (const T*)st_s(slot), (const T*)st_y(slot), sprev, stil, (const T*)pol_tr,
             (const T*)(pol_lr + j * m), pol_lr + (j + 1) * m, rho_in + (j + 1) * m, pol_Xr + j * m, Nr,
             pol_Jr + j * m, (const T*)pol_sc);
    enqueue_step_params(j + 1, st);
  }

  cosmo_status pol_forward(int32_t K_, const double* sigma, const void* tr, const void* ta, const void* l0,
                           const void* x0, const void* s0, const void* y0, void* xK, void* sK, void* yK, double* loss,
                           int32_t tape, cudaStream_t st) override {
    if (K_ < 1) return fail(COSMO_E_INVAL, "K must be >= 1");
    if (!tr || !ta || !l0) return fail(COSMO_E_INVAL, "theta_rho, theta_alpha and l0 are required");
    TRY(ensure_tape(K_));
    TRY(pol_alloc(K_));
    CU(cudaMemcpyAsync(pol_tr, tr, sizeof(T) * ws_nparams(POL_NFR, 1, POL_H), cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(pol_ta, ta, sizeof(T) * ws_nparams(POL_NFA, 1, POL_H), cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(pol_l0, l0, sizeof(T) * 5, cudaMemcpyDeviceToDevice, st));
    pol_mode = true;
    const cosmo_status r = forward(K_, sigma, nullptr, nullptr, x0, s0, y0, xK, sK, yK, loss, tape, st);
    pol_mode = false;
    pol_valid = r == COSMO_OK && tape != 0;
    return r;
  }

  cosmo_status pol_backward(const void* gx, const void* gs, const void* gy, const double* gl, void* gtr, void* gta,
                            void* gl0, void* gx0, void* gs0, void* gy0, cudaStream_t st) override {
    if (!pol_valid) return fail(COSMO_E_STATE, "policy backward needs a policy forward with record_tape=1");
    if (!gtr || !gta || !gl0) return fail(COSMO_E_INVAL, "gtheta_rho, gtheta_alpha and gl0 are required");
    TRY(backward(gx, gs, gy, gl, nullptr, nullptr, gx0, gs0, gy0, st));
    const int64_t m = h.m, ni = h.ninst, Nr = (int64_t)(K - 1) * m, Na = (int64_t)(K - 1) * ni;
    if (m > 0)
      launch("pol_bwd", k_pol_scan<T, false>, (int)((m + 255) / 256), 256, 0, st, K, m, (const T*)grho_all,
             (const T*)rho_in, (const T*)pol_lr, (const T*)pol_Jr, pol_Gr, pol_glr);
    launch("pol_bwd", k_pol_scan<T, true>, (int)((ni + 255) / 256), 256, 0, st, K, ni, (const T*)galpha_all,
           (const T*)alpha_in, (const T*)pol_la, (const T*)pol_Ja, pol_Ga, pol_gla);
    launch("pol_bwd", k_pol_l0<T, V>, 1, 256, 0, st, P, (const T*)pol_glr, (const T*)pol_gla, (T*)gl0);
    CU(cudaGetLastError());
    launched += 3; g_launches += 3;
    if (Nr == 0) TRY((mlp_bwd<POL_NFR, 1, POL_H>(0, pol_Xr, 0, pol_tr, pol_Gr, 0, (T*)gtr, 0, pol_h1, pol_d1,
                                                  pol_h2, pol_d2, pol_part, "pol_bwd", st)));
    for (int64_t e0 = 0; e0 < Nr; e0 += pol_ch)
      TRY((mlp_bwd<POL_NFR, 1, POL_H>(std::min(pol_ch, Nr - e0), pol_Xr + e0, Nr, pol_tr, pol_Gr + e0, Nr, (T*)gtr,
                                      e0 > 0, pol_h1, pol_d1, pol_h2, pol_d2, pol_part, "pol_bwd", st)));
    if (Na == 0) TRY((mlp_bwd<POL_NFA, 1, POL_H>(0, pol_Xa, 0, pol_ta, pol_Ga, 0, (T*)gta, 0, pol_h1, pol_d1,
                                                  pol_h2, pol_d2, pol_part, "pol_bwd", st)));
    for (int64_t e0 = 0; e0 < Na; e0 += pol_ch)
      TRY((mlp_bwd<POL_NFA, 1, POL_H>(std::min(pol_ch, Na - e0), pol_Xa + e0, Na, pol_ta, pol_Ga + e0, Na, (T*)gta,
                                      e0 > 0, pol_h1, pol_d1, pol_h2, pol_d2, pol_part, "pol_bwd", st)));
    return COSMO_OK;
  }

  cosmo_status pol_schedule(void* rho, void* alpha, cudaStream_t st) override {
    if (pol_K == 0 || K != pol_K) return fail(COSMO_E_STATE, "no policy forward");
    if (rho) CU(cudaMemcpyAsync(rho, rho_in, sizeof(T) * K * h.m, cudaMemcpyDeviceToDevice, st));
    if (alpha) CU(cudaMemcpyAsync(alpha, alpha_in, sizeof(T) * K * h.ninst, cudaMemcpyDeviceToDevice, st));
    return COSMO_OK;
  }

  cosmo_status residuals(const void* x, const void* s, const void* y, double* rp2, double* rd2,
                         double* obj, cudaStream_t st) override {
    if (!x || !s || !y) return fail(COSMO_E_INVAL, "x, s, y are required");
    ResArgs<T> ra{(const T*)x, (const T*)s, (const T*)y, nullptr, nullptr, rp2, rd2, obj, nullptr};
    seq_kernels = 0;
    launch("residuals", k_residuals<T, V, 256>, h.ninst, 256, 0, st, P, ra);
    CU(cudaGetLastError());
    launched += 1; g_launches += 1;
    return COSMO_OK;
  }

  cosmo_status rho_from_log(int32_t K_, const double* lr, double eq, void* rho, cudaStream_t st) override {
    if (K_ < 1 || K_ > 65535 || !lr || !rho) return fail(COSMO_E_INVAL, "bad arguments to rho_from_log");
    const dim3 grid(grid_for(h.m, 256, 148 * 4), K_);   // y: step
    k_rho_from_log<T, V><<<grid, 256, 0, st>>>(P, K_, lr, eq, (T*)rho);
    CU(cudaGetLastError());
    launched += 1; g_launches += 1;
    return COSMO_OK;
  }
  cosmo_status rho_from_log_bwd(int32_t K_, const void* rho, const void* grho, double* glog,
                                cudaStream_t st) override {
    if (K_ < 1 || !rho || !grho || !glog) return fail(COSMO_E_INVAL, "bad arguments to rho_from_log_backward");
    k_rowsum_prod<T, 256><<<K_, 256, 0, st>>>(h.m, (const T*)grho, (const T*)rho, glog);
    CU(cudaGetLastError());
    launched += 1; g_launches += 1;
    return COSMO_OK;
  }
  cosmo_status alpha_bcast(int32_t K_, const double* a, void* alpha, cudaStream_t st) override {
    if (K_ < 1 || !a || !alpha) return fail(COSMO_E_INVAL, "bad arguments to alpha_broadcast");
    k_broadcast<T><<<grid_for((int64_t)K_ * h.ninst, 256), 256, 0, st>>>(K_, h.ninst, a, (T*)alpha);
    CU(cudaGetLastError());
    launched += 1; g_launches += 1;
    return COSMO_OK;
  }
  cosmo_status alpha_reduce(int32_t K_, const void* ga, double* gk, cudaStream_t st) override {
    if (K_ < 1 || !ga || !gk) return fail(COSMO_E_INVAL, "bad arguments to alpha_reduce");
    k_rowsum_prod<T, 256><<<K_, 256, 0, st>>>(h.ninst, (const T*)ga, (const T*)nullptr, gk);
    CU(cudaGetLastError());
    launched += 1; g_launches += 1;
    return COSMO_OK;
  }
  cosmo_status flags_sync(int32_t* out) override {
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpy(out, flags, sizeof(int32_t) * h.ninst, cudaMemcpyDeviceToHost));
    CU(cudaMemset(flags, 0, sizeof(int32_t) * h.ninst));
    return COSMO_OK;
  }
  void info(cosmo_batch_info* o) const override {
    o->ninst = h.ninst;
    o->n_total = h.n;
    o->m_total = h.m;
    o->nnzA = (int64_t)h.A_ci.size();
    o->nnzP = (int64_t)h.P_ci.size();
    o->n_soc = (int32_t)h.soc_row0.size();
    o->n_psd = (int32_t)h.psd_p.size();
    o->max_psd_p = h.max_p;
    o->psd_u_entries = h.sum_p2;
    o->device_bytes = arena.bytes + (tape_external ? 0 : tarena.bytes) + sarena.bytes + warena.bytes + parena.bytes;
    o->last_K = K;
    o->tape_valid = tape_valid ? 1 : 0;
    o->kernels_launched = launched;
    o->fwd_persistent = persist_now() ? 1 : 0;
    unsigned long long st6[6] = {0, 0, 0, 0, 0, 0};
    if (cudaDeviceSynchronize() == cudaSuccess &&
        cudaMemcpy(st6, stats, sizeof(st6), cudaMemcpyDeviceToHost) == cudaSuccess) {
      o->eig_sweeps = (int64_t)st6[0];
      o->eig_blocks = (int64_t)st6[1];
      o->cg_iters = (int64_t)st6[2];
      o->cg_solves = (int64_t)st6[3];
      o->adj_cg_iters = (int64_t)st6[4];
      o->adj_cg_solves = (int64_t)st6[5];
    } else {
      cudaGetLastError();
    }
  }
};

// ------------------------------------------------------------------ ABI ---
extern "C" {

const char* cosmo_version(void) { return "cosmo_du 0.1 (sm_103a)"; }
int64_t cosmo_kernel_launch_count(void) { return g_launches.load(); }
const char* cosmo_last_error(void) { return g_err.c_str(); }

cosmo_status cosmo_options_default(cosmo_options* o, int32_t precision) {
  if (!o) return fail(COSMO_E_INVAL, "options pointer is NULL");
  if (precision != COSMO_PREC_MIXED && precision != COSMO_PREC_FP64)
    return fail(COSMO_E_INVAL, "unknown precision %d", precision);
  std::memset(o, 0, sizeof(*o));
  o->precision = precision;
  o->value_type = COSMO_VAL_F32;
  o->cg_tol = precision == COSMO_PREC_FP64 ? 1e-10 : 1e-8;
  o->cg_max_iter = 500;
  o->checkpoint_every = 0;
  o->dk_gap_tau = 1e-12;
  o->eig_jacobi_max_p = 0;
  o->eig_max_sweeps = 30;
  o->eig_tol = precision == COSMO_PREC_FP64 ? 1e-14 : 1e-6;
  o->use_graph = 1;
  o->device = 0;
  o->eig_warm_start = 1;
  o->dk_tensor_cores = 1;
  o->cg_cluster = 0;
  o->eig_variant = 0;
  o->eig_threads = 0;
  o->autotune = 0;
  o->fwd_persistent = 0;
  o->loss_kind = 0;
  return COSMO_OK;
}

cosmo_status cosmo_problem_validate(const cosmo_problem* prob) {
  g_err.clear();
  return validate(prob);
}

cosmo_status cosmo_batch_create(const cosmo_problem* prob, const cosmo_options* opt,
                                cosmo_batch** out) {
  g_err.clear();
  if (!out) return fail(COSMO_E_INVAL, "out is NULL");
  *out = nullptr;
  cosmo_options o;
  if (opt) o = *opt;
  else cosmo_options_default(&o, COSMO_PREC_MIXED);
  if (o.precision != COSMO_PREC_MIXED && o.precision != COSMO_PREC_FP64)
    return fail(COSMO_E_INVAL, "unknown precision %d", o.precision);
  if (o.value_type != COSMO_VAL_F32 && o.value_type != COSMO_VAL_BF16)
    return fail(COSMO_E_INVAL, "unknown value type %d", o.value_type);
  if (!(o.cg_tol > 0.0) || o.cg_max_iter < 1 || o.checkpoint_every < 0 || !(o.dk_gap_tau >= 0.0) ||
      o.eig_max_sweeps < 1 || !(o.eig_tol > 0.0) ||
      !(o.cg_cluster >= -4 && o.cg_cluster <= 4 && o.cg_cluster != 3) ||
      !(o.loss_kind == 0 || o.loss_kind == 1) || o.eig_variant < 0 || o.eig_variant > 3 ||
      !(o.autotune == 0 || o.autotune == 1) || !(o.fwd_persistent == 0 || o.fwd_persistent == 1) ||
      !(o.eig_threads == 0 || o.eig_threads == 128 || o.eig_threads == 256 || o.eig_threads == 512 ||
        (o.eig_threads == 1024 && o.eig_variant != 1)))
    return fail(COSMO_E_INVAL, "invalid options");
  TRY(validate(prob));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(COSMO_E_NODEVICE, "no CUDA device");
  }
  if (o.device < 0 || o.device >= ndev) return fail(COSMO_E_INVAL, "device %d out of range", o.device);
  CU(cudaSetDevice(o.device));
  std::unique_ptr<cosmo_batch> b(new cosmo_batch());
  b->opt = o;
  build_plan(prob, b->plan);
  cosmo_status st;
  if (o.precision == COSMO_PREC_FP64) {
    auto* im = new ImplT<double, double>(o, b->plan);
    b->impl.reset(im);
    st = im->init();
  } else if (o.value_type == COSMO_VAL_BF16) {
    auto* im = new ImplT<float, __nv_bfloat16>(o, b->plan);
    b->impl.reset(im);
    st = im->init();
  } else {
    auto* im = new ImplT<float, float>(o, b->plan);
    b->impl.reset(im);
    st = im->init();
  }
  if (st != COSMO_OK) return st;
  *out = b.release();
  return COSMO_OK;
}

cosmo_status cosmo_batch_destroy(cosmo_batch* b) {
  if (!b) return COSMO_OK;
  cudaSetDevice(b->opt.device);
  cudaDeviceSynchronize();
  delete b;
  return COSMO_OK;
}

cosmo_status cosmo_batch_get_tuning(const cosmo_batch* b, cosmo_tuning* out) {
  g_err.clear();
  if (!b || !out) return fail(COSMO_E_INVAL, "null argument");
  b->impl->get_tuning(out);
  return COSMO_OK;
}

cosmo_status cosmo_batch_set_tuning(cosmo_batch* b, const cosmo_tuning* t) {
  g_err.clear();
  if (!b || !t) return fail(COSMO_E_INVAL, "null argument");
  CU(cudaSetDevice(b->opt.device));
  return b->impl->set_tuning(*t);
}

cosmo_status cosmo_batch_get_info(const cosmo_batch* b, cosmo_batch_info* out) {
  if (!b || !out) return fail(COSMO_E_INVAL, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->precision = b->opt.precision;
  b->impl->info(out);
  return COSMO_OK;
}

#define BATCH_GUARD(b)                                           \
  do {                                                           \
    g_err.clear();                                               \
    if (!(b)) return fail(COSMO_E_INVAL, "batch is NULL");       \
    CU(cudaSetDevice((b)->opt.device));                          \
  } while (0)

cosmo_status cosmo_forward(cosmo_batch* b, int32_t K, const double* sigma_host, const void* rho,
                           const void* alpha, const void* x0, const void* s0, const void* y0,
                           void* xK, void* sK, void* yK, double* loss, int32_t record_tape,
                           void* stream) {
  BATCH_GUARD(b);
  return b->impl->forward(K, sigma_host, rho, alpha, x0, s0, y0, xK, sK, yK, loss, record_tape,
                          (cudaStream_t)stream);
}

cosmo_status cosmo_backward(cosmo_batch* b, const void* gxK, const void* gsK, const void* gyK,
                            const double* gloss, void* grho, void* galpha, void* gx0, void* gs0,
                            void* gy0, void* stream) {
  BATCH_GUARD(b);
  return b->impl->backward(gxK, gsK, gyK, gloss, grho, galpha, gx0, gs0, gy0, (cudaStream_t)stream);
}

cosmo_status cosmo_residuals(cosmo_batch* b, const void* x, const void* s, const void* y,
                             double* rp2, double* rd2, double* obj, void* stream) {
  BATCH_GUARD(b);
  return b->impl->residuals(x, s, y, rp2, rd2, obj, (cudaStream_t)stream);
}

cosmo_status cosmo_solve_params_default(cosmo_solve_params* p) {
  g_err.clear();
  if (!p) return fail(COSMO_E_INVAL, "p is NULL");
  p->sigma = 1e-6;
  p->alpha = 1.6;
  p->rho0 = 0.1;
  p->rho_eq_scale = 1e3;
  p->eps = 1e-3;
  p->rebalance_tol = 5.0;
  p->rho_min = 1e-6;
  p->rho_max = 1e6;
  p->max_iter = 5000;
  p->check_every = 25;
  p->rebalance_every = 25;
  p->pad = 0;
  return COSMO_OK;
}

cosmo_status cosmo_solve(cosmo_batch* b, const cosmo_solve_params* prm, void* x, void* s, void* y,
                         int32_t* iters, double* rbar_p, double* rbar_d, double* rho, void* stream) {
  BATCH_GUARD(b);
  if (!prm) return fail(COSMO_E_INVAL, "prm is NULL");
  return b->impl->solve(*prm, x, s, y, iters, rbar_p, rbar_d, rho, (cudaStream_t)stream);
}

cosmo_status cosmo_policy_sizes(int32_t* n_theta_rho, int32_t* n_theta_alpha) {
  if (!n_theta_rho || !n_theta_alpha) return fail(COSMO_E_INVAL, "NULL output");
  *n_theta_rho = ws_nparams(POL_NFR, 1, POL_H);
  *n_theta_alpha = ws_nparams(POL_NFA, 1, POL_H);
  return COSMO_OK;
}

cosmo_status cosmo_policy_forward(cosmo_batch* b, int32_t K, const double* sigma_host, const void* theta_rho,
                                  const void* theta_alpha, const void* l0, const void* x0, const void* s0,
                                  const void* y0, void* xK, void* sK, void* yK, double* loss, int32_t record_tape,
                                  void* stream) {
  BATCH_GUARD(b);
  return b->impl->pol_forward(K, sigma_host, theta_rho, theta_alpha, l0, x0, s0, y0, xK, sK, yK, loss, record_tape,
                              (cudaStream_t)stream);
}

cosmo_status cosmo_policy_backward(cosmo_batch* b, const void* gx, const void* gs, const void* gy,
                                   const double* gloss, void* gtheta_rho, void* gtheta_alpha, void* gl0, void* gx0,
                                   void* gs0, void* gy0, void* stream) {
  BATCH_GUARD(b);
  return b->impl->pol_backward(gx, gs, gy, gloss, gtheta_rho, gtheta_alpha, gl0, gx0, gs0, gy0,
                               (cudaStream_t)stream);
}

cosmo_status cosmo_policy_schedule(cosmo_batch* b, void* rho, void* alpha, void* stream) {
  BATCH_GUARD(b);
  return b->impl->pol_schedule(rho, alpha, (cudaStream_t)stream);
}

cosmo_status cosmo_ws_sizes(int32_t* n_theta_x, int32_t* n_theta_c) {
  if (!n_theta_x || !n_theta_c) return fail(COSMO_E_INVAL, "NULL output");
  *n_theta_x = ws_nparams(WS_NFX, 1);
  *n_theta_c = ws_nparams(WS_NFC, 2);
  return COSMO_OK;
}

cosmo_status cosmo_ws_forward(cosmo_batch* b, const void* theta_x, const void* theta_c, void* x0, void* s0,
                              void* y0, void* stream) {
  BATCH_GUARD(b);
  return b->impl->ws_forward(theta_x, theta_c, x0, s0, y0, (cudaStream_t)stream);
}

cosmo_status cosmo_ws_backward(cosmo_batch* b, const void* theta_x, const void* theta_c, const void* gx0,
                               const void* gs0, const void* gy0, void* gtheta_x, void* gtheta_c, void* stream) {
  BATCH_GUARD(b);
  return b->impl->ws_backward(theta_x, theta_c, gx0, gs0, gy0, gtheta_x, gtheta_c, (cudaStream_t)stream);
}

cosmo_status cosmo_rho_from_log(cosmo_batch* b, int32_t K, const double* log_rho, double eq_scale,
                                void* rho, void* stream) {
  BATCH_GUARD(b);
  return b->impl->rho_from_log(K, log_rho, eq_scale, rho, (cudaStream_t)stream);
}

cosmo_status cosmo_rho_from_log_backward(cosmo_batch* b, int32_t K, const void* rho,
                                         const void* grho, double* glog, void* stream) {
  BATCH_GUARD(b);
  return b->impl->rho_from_log_bwd(K, rho, grho, glog, (cudaStream_t)stream);
}

cosmo_status cosmo_alpha_broadcast(cosmo_batch* b, int32_t K, const double* alpha_k, void* alpha,
                                   void* stream) {
  BATCH_GUARD(b);
  return b->impl->alpha_bcast(K, alpha_k, alpha, (cudaStream_t)stream);
}

cosmo_status cosmo_alpha_reduce(cosmo_batch* b, int32_t K, const void* galpha, double* galpha_k,
                                void* stream) {
  BATCH_GUARD(b);
  return b->impl->alpha_reduce(K, galpha, galpha_k, (cudaStream_t)stream);
}

cosmo_status cosmo_profile_enable(cosmo_batch* b, const char* kernel) {
  BATCH_GUARD(b);
  return b->impl->profile_enable(kernel);
}

cosmo_status cosmo_profile_read(cosmo_batch* b, const char* kernel, double* total_ms,
                                int64_t* launches, int32_t reset) {
  BATCH_GUARD(b);
  if (!total_ms || !launches) return fail(COSMO_E_INVAL, "NULL output");
  return b->impl->profile_read(kernel, total_ms, launches, reset);
}

cosmo_status cosmo_workspace_bytes(const cosmo_batch* b, int32_t K, size_t* bytes) {
  g_err.clear();
  if (!b || !bytes) return fail(COSMO_E_INVAL, "null argument");
  if (K < 1) return fail(COSMO_E_INVAL, "K must be >= 1");
  *bytes = b->impl->workspace_bytes(K);
  return COSMO_OK;
}

cosmo_status cosmo_batch_set_workspace(cosmo_batch* b, int32_t K, void* ws, size_t bytes) {
  BATCH_GUARD(b);
  return b->impl->set_workspace_ext(K, ws, bytes);
}

cosmo_status cosmo_tape_eigen(cosmo_batch* b, int32_t k, void* lam, void* U, void* stream) {
  BATCH_GUARD(b);
  return b->impl->tape_eigen(k, lam, U, (cudaStream_t)stream);
}

cosmo_status cosmo_status_sync(cosmo_batch* b, int32_t* flags_host) {
  BATCH_GUARD(b);
  if (!flags_host) return fail(COSMO_E_INVAL, "flags_host is NULL");
  return b->impl->flags_sync(flags_host);
}



cosmo_status cosmo_step_host(cosmo_batch* b, int32_t K, double sigma, double eq_scale,
                             const double* lr_h, const double* ak_h, const void* x0_h,
                             const void* s0_h, const void* y0_h, double* loss_h, double* glr_h,
                             double* gak_h, void* gx0_h, void* gs0_h, void* gy0_h, void* stream) {
  BATCH_GUARD(b);
  if (K < 1 || !lr_h || !ak_h || !loss_h || !glr_h || !gak_h)
    return fail(COSMO_E_INVAL, "bad arguments to cosmo_step_host");
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->hostbufs) b->hostbufs.reset(new HostStepBufs());
  HostStepBufs* hb = b->hostbufs.get();
  const HostPlan& h = b->plan;
  const size_t rs = b->impl->real_size();
  if (hb->K != K) {
    CU(cudaDeviceSynchronize());
    hb->a.release();
    hb->K = K;
    char* p;
    TRY(hb->a.alloc(&hb->lr, K)); TRY(hb->a.alloc(&hb->ak, K)); TRY(hb->a.alloc(&hb->glr, K));
    TRY(hb->a.alloc(&hb->gak, K)); TRY(hb->a.alloc(&hb->loss, h.ninst));
    TRY(hb->a.alloc(&hb->gloss, h.ninst));
    TRY(hb->a.alloc(&p, (int64_t)rs * K * h.m)); hb->rho = p;
    TRY(hb->a.alloc(&p, (int64_t)rs * K * h.m)); hb->grho = p;
    TRY(hb->a.alloc(&p, (int64_t)rs * K * h.ninst)); hb->alpha = p;
    TRY(hb->a.alloc(&p, (int64_t)rs * K * h.ninst)); hb->galpha = p;
    TRY(hb->a.alloc(&p, (int64_t)rs * h.n)); hb->x0 = p;
    TRY(hb->a.alloc(&p, (int64_t)rs * h.m)); hb->s0 = p;
    TRY(hb->a.alloc(&p, (int64_t)rs * h.m)); hb->y0 = p;
    TRY(hb->a.alloc(&p, (int64_t)rs * h.n)); hb->gx0 = p;
    TRY(hb->a.alloc(&p, (int64_t)rs * h.m)); hb->gs0 = p;
    TRY(hb->a.alloc(&p, (int64_t)rs * h.m)); hb->gy0 = p;
    std::vector<double> ones(h.ninst, 1.0);
    CU(cudaMemcpy(hb->gloss, ones.data(), sizeof(double) * h.ninst, cudaMemcpyHostToDevice));
  }
  CU(cudaMemcpyAsync(hb->lr, lr_h, sizeof(double) * K, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(hb->ak, ak_h, sizeof(double) * K, cudaMemcpyHostToDevice, st));
  if (x0_h) CU(cudaMemcpyAsync(hb->x0, x0_h, rs * h.n, cudaMemcpyHostToDevice, st));
  if (s0_h) CU(cudaMemcpyAsync(hb->s0, s0_h, rs * h.m, cudaMemcpyHostToDevice, st));
  if (y0_h) CU(cudaMemcpyAsync(hb->y0, y0_h, rs * h.m, cudaMemcpyHostToDevice, st));
  TRY(b->impl->rho_from_log(K, hb->lr, eq_scale, hb->rho, st));
  TRY(b->impl->alpha_bcast(K, hb->ak, hb->alpha, st));
  std::vector<double> sg(K, sigma);
  TRY(b->impl->forward(K, sg.data(), hb->rho, hb->alpha, x0_h ? hb->x0 : nullptr,
                       s0_h ? hb->s0 : nullptr, y0_h ? hb->y0 : nullptr, nullptr, nullptr, nullptr,
                       hb->loss, 1, st));
  TRY(b->impl->backward(nullptr, nullptr, nullptr, hb->gloss, hb->grho, hb->galpha,
                        gx0_h ? hb->gx0 : nullptr, gs0_h ? hb->gs0 : nullptr,
                        gy0_h ? hb->gy0 : nullptr, st));
  TRY(b->impl->rho_from_log_bwd(K, hb->rho, hb->grho, hb->glr, st));
  TRY(b->impl->alpha_reduce(K, hb->galpha, hb->gak, st));
  CU(cudaMemcpyAsync(loss_h, hb->loss, sizeof(double) * h.ninst, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(glr_h, hb->glr, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(gak_h, hb->gak, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
  if (gx0_h) CU(cudaMemcpyAsync(gx0_h, hb->gx0, rs * h.n, cudaMemcpyDeviceToHost, st));
  if (gs0_h) CU(cudaMemcpyAsync(gs0_h, hb->gs0, rs * h.m, cudaMemcpyDeviceToHost, st));
  if (gy0_h) CU(cudaMemcpyAsync(gy0_h, hb->gy0, rs * h.m, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return COSMO_OK;
}

}  // extern "C"

// ---- standalone PSD kernels ----
template <class T>
static cosmo_status psd_project_t(int32_t nblk, const int32_t* p_h, const int64_t* off_h,
                                  const void* v, void* out, void* lam, void* U, cudaStream_t st) {
  // Jacobi for p <= 64, tridiagonal + QL above; two launches when mixed
  std::vector<int32_t> p(p_h, p_h + nblk);
  std::vector<int64_t> off(off_h, off_h + nblk), loff(nblk), uoff(nblk);
  int64_t sl = 0, su = 0;
  for (int32_t j = 0; j < nblk; ++j) {
    if (p[j] < 1 || p[j] > 1024) return fail(COSMO_E_INVAL, "PSD order out of range");
    loff[j] = sl; uoff[j] = su; sl += p[j]; su += (int64_t)p[j] * p[j];
  }
  int dev = 0, maxs = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  DevArena a;
  T* Uw = (T*)U;
  if (!Uw) TRY(a.alloc(&Uw, su));
  int32_t* dflag;
  TRY(a.alloc(&dflag, 1));
  CU(cudaMemsetAsync(dflag, 0, sizeof(int32_t), st));
  const double tol = sizeof(T) == 8 ? 1e-14 : 1e-6;
  for (int method = 0; method < 2; ++method) {
    std::vector<int32_t> pp;
    std::vector<int64_t> oo, lo, uo;
    int maxp = 0;
    for (int32_t j = 0; j < nblk; ++j)
      if ((p[j] > 64) == (method == 1)) {
        pp.push_back(p[j]); oo.push_back(off[j]); lo.push_back(loff[j]); uo.push_back(uoff[j]);
        maxp = std::max(maxp, p[j]);
      }
    if (pp.empty()) continue;
    int32_t* dp;
    int64_t *doff, *dloff, *duoff;
    TRY(a.upload(&dp, pp)); TRY(a.upload(&doff, oo)); TRY(a.upload(&dloff, lo)); TRY(a.upload(&duoff, uo));
    PsdBatch<T> B{(int32_t)pp.size(), dp, doff, dloff, duoff};
    if (method == 0) {
      const size_t smem = psd_fwd_smem<T>(maxp, 256);
      if ((int64_t)smem > maxs) return fail(COSMO_E_INVAL, "PSD order %d too large for one CTA", maxp);
      CU(cudaFuncSetAttribute(k_psd_project_batch<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_psd_project_batch<T, 256><<<B.nblk, 256, smem, st>>>(B, (const T*)v, (T*)out, (T*)lam, Uw, tol, 30, dflag);
    } else {
      const size_t smem = tql_smem<T>(maxp, 256);
      CU(cudaFuncSetAttribute(k_psd_project_tql<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_psd_project_tql<T, 256><<<B.nblk, 256, smem, st>>>(B, (const T*)v, (T*)out, (T*)lam, Uw, 120, dflag);
    }
    CU(cudaGetLastError());
    g_launches += 1;
  }
  CU(cudaStreamSynchronize(st));
  return COSMO_OK;
}

template <class T>
static cosmo_status psd_dk_t(int32_t nblk, const int32_t* p_h, const int64_t* off_h,
                             const void* lam, const void* U, const void* g, void* out, double tau,
                             cudaStream_t st) {
  std::vector<int32_t> p(p_h, p_h + nblk);
  std::vector<int64_t> off(off_h, off_h + nblk), loff(nblk), uoff(nblk);
  int64_t sl = 0, su = 0;
  int maxp = 0;
  for (int32_t j = 0; j < nblk; ++j) {
    if (p[j] < 1 || p[j] > 1024) return fail(COSMO_E_INVAL, "PSD order out of range");
    loff[j] = sl; uoff[j] = su; sl += p[j]; su += (int64_t)p[j] * p[j];
    maxp = std::max(maxp, p[j]);
  }
  const size_t smem = psd_bwd_smem<T>(maxp, 256);
  int dev = 0, maxs = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if ((int64_t)smem > maxs) return fail(COSMO_E_INVAL, "PSD order %d too large for one CTA", maxp);
  CU(cudaFuncSetAttribute(k_psd_dk_batch<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DevArena a;
  int32_t* dp;
  int64_t *doff, *dloff, *duoff;
  TRY(a.upload(&dp, p)); TRY(a.upload(&doff, off)); TRY(a.upload(&dloff, loff)); TRY(a.upload(&duoff, uoff));
  PsdBatch<T> B{nblk, dp, doff, dloff, duoff};
  if constexpr (std::is_same<T, float>::value) {
    if (maxp <= DK_TC_MAXP) {
      // tensor-core path (the default of the batched backward for these orders)
      int32_t* err;
      TRY(a.alloc(&err, 1));
      CU(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
      const size_t tsm = dk_tc_smem(maxp);
      CU(cudaFuncSetAttribute(k_psd_dk_batch_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
      k_psd_dk_batch_tc<<<nblk, DK_TC_NT, tsm, st>>>(B, (const float*)lam, (const float*)U, (const float*)g,
                                                     (float*)out, tau, err);
      CU(cudaGetLastError());
      g_launches += 1;
      int32_t herr = 0;
      CU(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      if (herr) return fail(COSMO_E_TIMEOUT, "tensor-core DK backward: a bounded wait gave up");
      return COSMO_OK;
    }
  }
  k_psd_dk_batch<T, 256><<<nblk, 256, smem, st>>>(B, (const T*)lam, (const T*)U, (const T*)g, (T*)out, tau);
  CU(cudaGetLastError());
  g_launches += 1;
  CU(cudaStreamSynchronize(st));
  return COSMO_OK;
}

// ---- standalone reduced-system solve ----
template <class T>
static cosmo_status pcg_solve_t(int32_t ninst, int64_t n, int64_t m, const int64_t* col_off,
                                const int64_t* row_off, const int64_t* A_rp, const int32_t* A_ci,
                                const void* A_v, const int64_t* AT_rp, const int32_t* AT_ci,
                                const void* AT_v, const int64_t* P_rp, const int32_t* P_ci,
                                const void* P_v, double sigma, const void* rho, const void* rhs,
                                void* x, int32_t warm, double tol, int32_t maxit, int32_t* iters,
                                cudaStream_t st) {
  const size_t bytes = sizeof(T) * (size_t)(4 * n + m) + sizeof(int32_t) * 2 * (size_t)ninst + 256;
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, bytes, st);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(COSMO_E_NOMEM, "workspace allocation failed: %s", cudaGetErrorString(e)); }
  T* dinv = reinterpret_cast<T*>(ws);
  T* r = dinv + n;
  T* p = r + n;
  T* u = p + n;
  T* t = u + n;
  int32_t* flags = reinterpret_cast<int32_t*>(t + m);
  int32_t* sched = flags + ninst;
  Prob<T, T> P{};
  P.ninst = ninst; P.n_total = n; P.m_total = m; P.col_off = col_off; P.row_off = row_off;
  P.A_rp = A_rp; P.A_ci = A_ci; P.A_v = (const T*)A_v;
  P.AT_rp = AT_rp; P.AT_ci = AT_ci; P.AT_v = (const T*)AT_v;
  P.P_rp = P_rp; P.P_ci = P_ci; P.P_v = (const T*)P_v;
  P.inst_sched = sched;
  cudaMemsetAsync(flags, 0, sizeof(int32_t) * ninst, st);
  k_iota<<<grid_for(ninst, 256), 256, 0, st>>>(ninst, sched);
  k_precond_csr<T, T><<<grid_for(n, 256), 256, 0, st>>>(P, sigma, (const T*)rho, dinv);
  CgArgs<T> ca{};
  ca.rhs = (const T*)rhs; ca.x = (T*)x; ca.x0 = nullptr; ca.rho = (const T*)rho; ca.dinv = dinv;
  ca.sigma = sigma; ca.r = r; ca.p = p; ca.u = u; ca.t = t; ca.tol = tol; ca.maxit = maxit;
  ca.zero_start = warm ? 0 : 1; ca.flag_bit = F_CG_CAP; ca.flags = flags; ca.iters = iters;
  k_pcg<T, T, 256><<<ninst, 256, 0, st>>>(P, ca);
  e = cudaGetLastError();
  cudaFreeAsync(ws, st);
  if (e != cudaSuccess) return fail(COSMO_E_CUDA, "pcg launch failed: %s", cudaGetErrorString(e));
  g_launches += 3;
  return COSMO_OK;
}

// Grid-wide CG (zero start) for large instances that no streamed plan
// takes: column / row tiles spread over the SMs, three kernels per iteration
// gathering from global memory, convergence read back every 8 iterations (the
// call synchronises the stream on this path).
template <class T>
static cosmo_status pcg_solve_grid_t(int32_t ninst, int64_t n, int64_t m, const int64_t* col_off_d,
                                     const int64_t* row_off_d, const Prob<T, T>& P0, double sigma,
                                     const void* rho, const void* rhs, void* x, double tol,
                                     int32_t maxit, int32_t* iters, cudaStream_t st) {
  std::vector<int64_t> co(ninst + 1), ro(ninst + 1), prp;
  int64_t nnz_a = 0;
  CU(cudaMemcpyAsync(co.data(), col_off_d, sizeof(int64_t) * (ninst + 1), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(ro.data(), row_off_d, sizeof(int64_t) * (ninst + 1), cudaMemcpyDeviceToHost, st));
  if (P0.P_rp) {
    prp.resize(n + 1);
    CU(cudaMemcpyAsync(prp.data(), P0.P_rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
  }
  if (m > 0) CU(cudaMemcpyAsync(&nnz_a, P0.A_rp + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  // P rows of at most 16 entries take one thread per row in the cols phase
  int short_p = 1;
  for (int64_t j = 0; j + 1 < (int64_t)prp.size() && short_p; ++j) short_p = prp[j + 1] - prp[j] <= 16;
  const int64_t nnz_p = prp.empty() ? 0 : prp[n];
  // batch width of the row routine from the mean row length; scalar loads
  // when an array is not 16-byte aligned
  auto aligned = [](const void* p, const void* q) {
    return ((uintptr_t)p % 16 == 0) && ((uintptr_t)q % 16 == 0);
  };
  auto vq_for = [](int64_t nnz, int64_t rows) {
    const int64_t mean = rows > 0 ? nnz / rows : 0;
    return mean >= 384 ? 4 : mean >= 128 ? 2 : 1;
  };
  int dev = 0, nsm = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

  DevArena a;
  // 256-thread CTAs gathering from global memory, tiles sized for about four
  // resident CTAs per SM (a multiple of 8, at most 256).
  auto tile_global = [&](int64_t total) {
    int64_t t = (total + 4 * nsm - 1) / (4 * nsm);
    t = (t + 7) / 8 * 8;
    return std::min<int64_t>(std::max<int64_t>(t, 8), 256);
  };
  const int64_t RTILE = tile_global(m), CTILE = tile_global(n);

  std::vector<int32_t> ct_inst, rt_inst, it_lo(ninst), it_hi(ninst), rt_first;
  std::vector<int64_t> ct_lo, ct_hi, rt_lo, rt_hi;
  for (int32_t i = 0; i < ninst; ++i) {
    it_lo[i] = (int32_t)ct_inst.size();
    for (int64_t c = co[i]; c < co[i + 1]; c += CTILE) {
      ct_inst.push_back(i); ct_lo.push_back(c); ct_hi.push_back(std::min(co[i + 1], c + CTILE));
    }
    it_hi[i] = (int32_t)ct_inst.size();
    // a row tile per instance (possibly empty): it records the iteration count
    bool first = true;
    for (int64_t q = ro[i]; q < ro[i + 1] || first; q += RTILE) {
      rt_inst.push_back(i); rt_lo.push_back(q); rt_hi.push_back(std::min(ro[i + 1], q + RTILE));
      rt_first.push_back(first ? 1 : 0);
      first = false;
      if (ro[i + 1] <= q) break;
    }
  }
  if (ct_inst.empty()) return COSMO_OK;
  GcgTiles G{};
  int32_t *d_ct_inst, *d_it_lo, *d_it_hi, *d_rt_inst = nullptr, *d_rt_first = nullptr;
  int64_t *d_ct_lo, *d_ct_hi, *d_rt_lo = nullptr, *d_rt_hi = nullptr;
  TRY(a.upload(&d_ct_inst, ct_inst)); TRY(a.upload(&d_ct_lo, ct_lo)); TRY(a.upload(&d_ct_hi, ct_hi));
  TRY(a.upload(&d_it_lo, it_lo)); TRY(a.upload(&d_it_hi, it_hi));
  if (!rt_inst.empty()) {
    TRY(a.upload(&d_rt_inst, rt_inst)); TRY(a.upload(&d_rt_lo, rt_lo)); TRY(a.upload(&d_rt_hi, rt_hi));
    TRY(a.upload(&d_rt_first, rt_first));
  }
  G.nct = (int32_t)ct_inst.size(); G.ct_inst = d_ct_inst; G.ct_lo = d_ct_lo; G.ct_hi = d_ct_hi;
  G.it_lo = d_it_lo; G.it_hi = d_it_hi;
  G.nrt = (int32_t)rt_inst.size(); G.rt_inst = d_rt_inst; G.rt_lo = d_rt_lo; G.rt_hi = d_rt_hi;
  G.rt_first = d_rt_first;
  G.nnz_a = nnz_a; G.nnz_p = nnz_p;
  G.vq_a = aligned(P0.A_ci, P0.A_v) ? vq_for(nnz_a, m) : 0;
  G.vq_at = aligned(P0.AT_ci, P0.AT_v) ? vq_for(nnz_a, n) : 0;
  G.vq_p = P0.P_rp && aligned(P0.P_ci, P0.P_v) ? vq_for(nnz_p, n) : 0;
  Prob<T, T> P = P0;
  T* dinv;
  TRY(a.alloc(&dinv, n));
  k_precond_csr<T, T><<<grid_for(n, 256), 256, 0, st>>>(P, sigma, (const T*)rho, dinv);
  ++g_launches;

  using T2 = typename Vec2<T>::type;
  GcgState<T> S{};
  T *rr, *uu, *tt;
  T2* zp;
  TRY(a.alloc(&rr, n)); TRY(a.alloc(&uu, n)); TRY(a.alloc(&zp, n));
  TRY(a.alloc(&tt, std::max<int64_t>(m, 1)));
  double *pa, *pb, *sc_rz, *sc_beta, *sc_alpha, *sc_bb;
  int32_t *cnt_grp, *cnt_inst, *sc_state, *running;
  TRY(a.alloc(&pa, G.nct)); TRY(a.alloc(&pb, G.nct));
  TRY(a.alloc(&sc_rz, 2 * ninst)); TRY(a.alloc(&sc_beta, 2 * ninst)); TRY(a.alloc(&sc_state, 2 * ninst));
  TRY(a.alloc(&sc_alpha, ninst)); TRY(a.alloc(&sc_bb, ninst));
  TRY(a.alloc(&cnt_grp, G.nct)); TRY(a.alloc(&cnt_inst, ninst));
  TRY(a.alloc(&running, maxit + 1));
  CU(cudaMemsetAsync(cnt_grp, 0, sizeof(int32_t) * G.nct, st));
  CU(cudaMemsetAsync(cnt_inst, 0, sizeof(int32_t) * ninst, st));
  CU(cudaMemsetAsync(running, 0, sizeof(int32_t) * (maxit + 1), st));
  S.rhs = (const T*)rhs; S.x = (T*)x; S.rho = (const T*)rho; S.dinv = dinv; S.sigma = sigma;
  S.r = rr; S.zp = zp; S.u = uu; S.t = tt; S.part_a = pa; S.part_b = pb; S.cnt_grp = cnt_grp; S.cnt_inst = cnt_inst;
  S.sc_rz = sc_rz; S.sc_beta = sc_beta; S.sc_state = sc_state; S.sc_alpha = sc_alpha; S.sc_bb = sc_bb;
  S.iters = iters; S.running = running; S.tol = tol; S.maxit = maxit;
  const size_t cols_smem_bytes = (size_t)CTILE * sizeof(T);
  k_gcg_init<T><<<G.nct, GCG_NT, 0, st>>>(G, S);
  ++g_launches;
  int32_t* h_run = nullptr;
  CU(cudaMallocHost(&h_run, sizeof(int32_t)));
  cosmo_status status = COSMO_OK;
  for (int it = 0; it <= maxit; ++it) {
    k_gcg_rows<T><<<G.nrt, GCG_NT, 0, st>>>(P, G, S, it);
    ++g_launches;
    if (it == maxit) break;   // the rows kernel at maxit records the capped counts
    k_gcg_cols<T><<<G.nct, GCG_NT, cols_smem_bytes, st>>>(P, G, S, it, short_p);
    k_gcg_update<T><<<G.nct, GCG_NT, 0, st>>>(P, G, S, it);
    g_launches += 2;
    if ((it & 7) == 7) {
      // instances still running at this iteration (counted by its rows kernel)
      cudaMemcpyAsync(h_run, running + it, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { status = fail(COSMO_E_CUDA, "grid CG failed: %s", cudaGetErrorString(e)); break; }
      if (*h_run == 0) {
        k_gcg_rows<T><<<G.nrt, GCG_NT, 0, st>>>(P, G, S, it + 1);   // records iteration counts
        ++g_launches;
        break;
      }
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess && status == COSMO_OK) status = fail(COSMO_E_CUDA, "grid CG launch failed: %s", cudaGetErrorString(e));
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && status == COSMO_OK) status = fail(COSMO_E_CUDA, "grid CG failed: %s", cudaGetErrorString(e));
  cudaFreeHost(h_run);
  return status;
}

// ---------------------------------------------------------------------------
// Prepared grid-wide solves (cosmo_pcg_plan): streaming layouts of A and A',
// tiles, workspace and the cooperative launch of k_gcg_stream.
// ---------------------------------------------------------------------------
struct PcgPlanBase {
  virtual ~PcgPlanBase() {}
  virtual cosmo_status solve(double sigma, const void* rho, const void* rhs, void* x, double tol,
                             int32_t maxit, int32_t* iters, cudaStream_t st) = 0;
  virtual void info(cosmo_pcg_plan_info* out) const = 0;
  virtual cosmo_status set_timing(int enable) = 0;
  virtual void get_timing(double* mean_us, double* slowest_us) const = 0;
};

// Contiguous tiles of the items [off[i], off[i+1]) of every instance, at
// most K in all, never crossing an instance; item j weighs rp[j+1] - rp[j] + 1
// (its entries, plus one).  Instances get tiles in proportion to their weight
// (at least one each when non-empty), and an instance's tiles have about
// equal weight.
static void gcs_tiles(const std::vector<int64_t>& off, const std::vector<int64_t>& rp, int K,
                      std::vector<int32_t>& inst, std::vector<int64_t>& lo, std::vector<int64_t>& hi,
                      std::vector<int32_t>* first_tile, std::vector<int32_t>* end_tile, int64_t& maxlen) {
  const int ni = (int)off.size() - 1;
  auto W = [&](int64_t a, int64_t b) { return (double)(rp[b] - rp[a]) + (double)(b - a); };
  const double tot = W(off[0], off[ni]);
  std::vector<int64_t> k(ni, 0);
  int64_t used = 0;
  for (int i = 0; i < ni; ++i) {
    const int64_t len = off[i + 1] - off[i];
    if (len <= 0) continue;
    k[i] = std::min<int64_t>(len, std::max<int64_t>(1, (int64_t)std::floor(K * W(off[i], off[i + 1]) / tot)));
    used += k[i];
  }
  while (used > K) {   // only the at-least-one rule can overshoot
    int best = -1;
    for (int i = 0; i < ni; ++i)
      if (k[i] > 1 && (best < 0 || k[i] > k[best])) best = i;
    if (best < 0) break;
    --k[best];
    --used;
  }
  while (used < K) {   // one more tile to the instance with the heaviest tiles
    int best = -1;
    double bw = 0.0;
    for (int i = 0; i < ni; ++i) {
      if (k[i] == 0 || k[i] >= off[i + 1] - off[i]) continue;
      const double w = W(off[i], off[i + 1]) / (double)k[i];
      if (best < 0 || w > bw) { best = i; bw = w; }
    }
    if (best < 0) break;
    ++k[best];
    ++used;
  }
  maxlen = 0;
  for (int i = 0; i < ni; ++i) {
    if (first_tile) (*first_tile)[i] = (int32_t)inst.size();
    const int64_t a = off[i], b = off[i + 1];
    int64_t prev = a, j = a;
    const double wi = W(a, b);
    for (int64_t q = 1; q < k[i]; ++q) {
      const double target = wi * (double)q / (double)k[i];
      while (j < b && W(a, j) < target) ++j;
      const int64_t cut = std::min(std::max(j, prev + 1), b - (k[i] - q));
      inst.push_back(i); lo.push_back(prev); hi.push_back(cut);
      maxlen = std::max(maxlen, cut - prev);
      prev = cut;
    }
    if (k[i] > 0) {
      inst.push_back(i); lo.push_back(prev); hi.push_back(b);
      maxlen = std::max(maxlen, b - prev);
    }
    if (end_tile) (*end_tile)[i] = (int32_t)inst.size();
  }
}

template <class T>
struct GcsPlan : PcgPlanBase {
  int32_t ninst = 0;
  int64_t n = 0, m = 0;
  DevArena a;
  Prob<T, T> P{};
  GcgTiles G{};
  GcsArgs<T> S{};
  int grid = 0, device = 0, cs = 1, nslot = 3, c_split = 0;
  int64_t layout_bytes = 0, quads_r = 0, quads_c = 0;
  unsigned* bar = nullptr;
  int32_t* h_err = nullptr;   // pinned
  // phase timer (off unless set_timing): stamps of the first kTsIters
  // iterations, and the last solve's per-phase means / slowest CTA
  static constexpr int kTsIters = 64;
  unsigned long long* ts = nullptr;
  double ph_mean[COSMO_PCG_PHASES] = {}, ph_max[COSMO_PCG_PHASES] = {};

  ~GcsPlan() override {
    if (h_err) cudaFreeHost(h_err);
  }

  // streaming layout of `rows` source rows (CSR rp/ci/v) cut into nseg
  // segments of each row's instance range in the gathered space gath_off;
  // the last row of each tile (tile_hi: one past the tiles' last rows) is
  // padded so that every tile's piece of a segment is whole chunks
  cosmo_status build_layout(int64_t rows, const int64_t* rp, const int32_t* ci, const T* v,
                            const int64_t* d_row_inst_off, const int64_t* d_gath_off, int nseg,
                            const std::vector<int64_t>& tile_hi, GcsLayout<T>& L, int64_t& quads,
                            cudaStream_t st) {
    constexpr int64_t CQ = gcs_cq<T>();
    L.nseg = nseg;
    L.rows = rows;
    std::vector<int64_t> qp((size_t)nseg * (rows + 1), 0);
    std::vector<char> last(rows > 0 ? rows : 1, 0);
    for (int64_t e : tile_hi)
      if (e > 0) last[e - 1] = 1;
    int64_t base = 0;
    if (rows > 0) {
      int32_t* cnt;
      TRY(a.alloc(&cnt, (int64_t)nseg * rows));
      k_gcs_count<<<(int)((rows * 32 + 255) / 256), 256, 0, st>>>(rows, rp, ci, ninst, d_row_inst_off,
                                                                  d_gath_off, nseg, cnt);
      ++g_launches;
      std::vector<int32_t> hc((size_t)nseg * rows);
      CU(cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * hc.size(), cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      for (int h = 0; h < nseg; ++h) {
        for (int64_t r = 0; r < rows; ++r) {
          qp[(size_t)h * (rows + 1) + r] = base;
          base += (hc[(size_t)h * rows + r] + 3) / 4;
          if (last[r]) base = (base + CQ - 1) / CQ * CQ;
        }
        qp[(size_t)h * (rows + 1) + rows] = base;
      }
    }
    if (base % CQ) return fail(COSMO_E_INVAL, "streamed CG plan: rows outside every tile");
    int64_t* d_qp;
    TRY(a.upload(&d_qp, qp));
    unsigned char* data = nullptr;
    if (base > 0) {
      TRY(a.alloc(&data, base / CQ * gcs_chunk_bytes<T>()));
      k_gcs_scatter<T><<<(int)((rows * 32 + 255) / 256), 256, 0, st>>>(rows, rp, ci, v, ninst, d_row_inst_off,
                                                                       d_gath_off, nseg, d_qp, data);
      ++g_launches;
    }
    L.data = data;
    L.qp = d_qp;
    quads = base;
    layout_bytes += base / CQ * gcs_chunk_bytes<T>() + (int64_t)qp.size() * 8;
    return COSMO_OK;
  }

  cosmo_status build(int32_t ninst_, int64_t n_, int64_t m_, const int64_t* col_off, const int64_t* row_off,
                     const int64_t* A_rp, const int32_t* A_ci, const T* A_v, const int64_t* AT_rp,
                     const int32_t* AT_ci, const T* AT_v, const int64_t* P_rp, const int32_t* P_ci,
                     const T* P_v, cudaStream_t st) {
    ninst = ninst_;
    n = n_;
    m = m_;
    int nsm = 0, optin = 0;
    CU(cudaGetDevice(&device));
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    if (ninst < 1 || ninst > nsm) return fail(COSMO_E_INVAL, "streamed CG plan: %d instances, at most %d", ninst, nsm);
    std::vector<int64_t> co(ninst + 1), ro(ninst + 1), arp(m + 1), atrp(n + 1), prp;
    CU(cudaMemcpyAsync(co.data(), col_off, sizeof(int64_t) * (ninst + 1), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(ro.data(), row_off, sizeof(int64_t) * (ninst + 1), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(arp.data(), A_rp, sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(atrp.data(), AT_rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    if (P_rp) {
      prp.resize(n + 1);
      CU(cudaMemcpyAsync(prp.data(), P_rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    }
    CU(cudaStreamSynchronize(st));
    auto monotone = [](const std::vector<int64_t>& v, int64_t last) {
      if (v.empty() || v[0] != 0 || v.back() != last) return false;
      for (size_t i = 1; i < v.size(); ++i)
        if (v[i] < v[i - 1]) return false;
      return true;
    };
    if (!monotone(co, n) || !monotone(ro, m) || !monotone(arp, arp.back()) || !monotone(atrp, arp.back()) ||
        (P_rp && !monotone(prp, prp.back())))
      return fail(COSMO_E_INVAL, "streamed CG plan: inconsistent offsets or row pointers");
    const int64_t nnz_a = arp.back(), nnz_p = P_rp ? prp.back() : 0;

    // plan-owned copies of the offsets and of P
    int64_t *d_co, *d_ro;
    TRY(a.upload(&d_co, co));
    TRY(a.upload(&d_ro, ro));
    P.ninst = ninst; P.n_total = n; P.m_total = m; P.col_off = d_co; P.row_off = d_ro;
    int short_p = 1, p_diag = 1;
    T* pd_dev = nullptr;
    if (P_rp) {
      int64_t* prp_d;
      int32_t* pci_d = nullptr;
      T* pv_d = nullptr;
      TRY(a.upload(&prp_d, prp));
      TRY(a.alloc(&pci_d, nnz_p));
      TRY(a.alloc(&pv_d, nnz_p));
      if (nnz_p > 0) {
        CU(cudaMemcpyAsync(pci_d, P_ci, sizeof(int32_t) * nnz_p, cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(pv_d, P_v, sizeof(T) * nnz_p, cudaMemcpyDeviceToDevice, st));
      }
      P.P_rp = prp_d; P.P_ci = pci_d; P.P_v = pv_d;
      for (int64_t j = 0; j < n && short_p; ++j) short_p = prp[j + 1] - prp[j] <= 16;
      // diagonal: every row holds at most its diagonal entry
      std::vector<int32_t> pci(nnz_p);
      if (nnz_p > 0) CU(cudaMemcpy(pci.data(), P_ci, sizeof(int32_t) * nnz_p, cudaMemcpyDeviceToHost));
      p_diag = 1;
      for (int64_t j = 0; j < n && p_diag; ++j)
        p_diag = prp[j + 1] - prp[j] == 0 || (prp[j + 1] - prp[j] == 1 && pci[prp[j]] == j);
      if (p_diag) {   // P_jj as a dense vector (0 for an empty row)
        std::vector<T> pv(nnz_p), pdh(n, T(0));
        if (nnz_p > 0) CU(cudaMemcpy(pv.data(), P_v, sizeof(T) * nnz_p, cudaMemcpyDeviceToHost));
        for (int64_t j = 0; j < n; ++j)
          if (prp[j + 1] > prp[j]) pdh[j] = pv[prp[j]];
        TRY(a.upload(&pd_dev, pdh));
      }
    }

    int64_t max_n = 0, max_m = 0;
    for (int i = 0; i < ninst; ++i) {
      max_n = std::max(max_n, co[i + 1] - co[i]);
      max_m = std::max(max_m, ro[i + 1] - ro[i]);
    }

    // cluster size CS (segments of z and t, one per CTA of a cluster) and
    // ring depth: the smallest CS whose stage, tables and a ring of at least
    // four chunks per warp fit shared memory (three if none does); tiles per
    // cluster, as many clusters as the device keeps resident
    const int64_t E = 16 / (int64_t)sizeof(T);
    std::vector<int32_t> rt_inst, ct_inst, it_lo(ninst), it_hi(ninst), irt_lo(ninst), irt_hi(ninst);
    std::vector<int64_t> rt_lo, rt_hi, ct_lo, ct_hi;
    GcsSmem sm{};
    int64_t RT = 0, CT = 0;
    auto make_tiles = [&](int K) {
      rt_inst.clear(); rt_lo.clear(); rt_hi.clear(); ct_inst.clear(); ct_lo.clear(); ct_hi.clear();
      gcs_tiles(ro, arp, K, rt_inst, rt_lo, rt_hi, &irt_lo, &irt_hi, RT);
      gcs_tiles(co, atrp, K, ct_inst, ct_lo, ct_hi, &it_lo, &it_hi, CT);
    };
    // R stages one segment of z; C the whole t (split 0) or one segment (1)
    auto smem_for = [&](int c, int ns, int64_t rt, int64_t ct, int split) {
      const int64_t stage_len = std::max((max_n + c - 1) / c, split ? (max_m + c - 1) / c : max_m) + 2 * E;
      const int64_t cto = std::max<int64_t>((ct + c - 1) / c, 1);
      return gcs_smem<T>(ns, stage_len, std::max<int64_t>(rt, 1), split ? std::max<int64_t>(ct, 1) : cto,
                         std::max<int64_t>((rt + c - 1) / c, 1), cto, ninst);
    };
    cs = 0;
    for (int want = 4; want >= 3 && !cs; --want) {
      for (int c : {1, 2, 4, 8}) {
        if (nsm / c < ninst) break;
        cudaFuncAttributes fa{};
        CU(cudaFuncGetAttributes(&fa, gcs_kernel(c)));
        const int64_t cap = (int64_t)optin - (int64_t)fa.sharedSizeBytes;
        make_tiles(nsm / c);
        for (int split = 0; split < 2 && !cs; ++split)
          for (int ns = GCS_MAXSLOT; ns >= want; --ns) {
            const GcsSmem t = smem_for(c, ns, RT, CT, split);
            if (t.total <= cap) { cs = c; nslot = ns; sm = t; c_split = split; break; }
          }
        if (cs) break;
      }
    }
    if (!cs) return fail(COSMO_E_INVAL, "streamed CG plan: the instances do not fit shared memory");
    const void* kern = gcs_kernel(cs);
    CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm.total));
    if (cs > 1) CU(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, cs > 8 ? 1 : 0));
    int ncl = 0;
    {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(nsm / cs * cs);
      cfg.blockDim = dim3(GCS_NT);
      cfg.dynamicSmemBytes = (size_t)sm.total;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      CU(cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg));
    }
    ncl = std::min(ncl, nsm / cs);
    if (ncl < ninst) return fail(COSMO_E_INVAL, "streamed CG plan: %d resident clusters for %d instances", ncl, ninst);
    if (ncl < nsm / cs) {
      // fewer resident clusters: larger tiles, so the deepest ring that still fits
      cudaFuncAttributes fa{};
      CU(cudaFuncGetAttributes(&fa, kern));
      const int64_t cap = (int64_t)optin - (int64_t)fa.sharedSizeBytes;
      make_tiles(ncl);
      for (nslot = GCS_MAXSLOT; nslot >= 2; --nslot) {
        sm = smem_for(cs, nslot, RT, CT, c_split);
        if (sm.total <= cap) break;
      }
      if (nslot < 2) return fail(COSMO_E_INVAL, "streamed CG plan: the instances do not fit shared memory");
      CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm.total));
    }
    if (ct_inst.empty()) return fail(COSMO_E_INVAL, "streamed CG plan: no columns");

    // streaming layouts: A by column segment (one per CTA of a cluster),
    // A' whole, its tiles the CTAs' shares of the cluster tiles' columns
    std::vector<int64_t> own_hi;
    for (size_t i = 0; i < ct_lo.size(); ++i) {
      const int64_t len = ct_hi[i] - ct_lo[i];
      for (int q = 1; q <= cs; ++q) own_hi.push_back(ct_lo[i] + len * q / cs);
    }
    TRY(build_layout(m, A_rp, A_ci, A_v, d_ro, d_co, cs, rt_hi, S.LR, quads_r, st));
    if (c_split) TRY(build_layout(n, AT_rp, AT_ci, AT_v, d_co, d_ro, cs, ct_hi, S.LC, quads_c, st));
    else TRY(build_layout(n, AT_rp, AT_ci, AT_v, d_co, d_ro, 1, own_hi, S.LC, quads_c, st));

    int32_t *d_ct_inst, *d_rt_inst = nullptr;
    int64_t *d_ct_lo, *d_ct_hi, *d_rt_lo = nullptr, *d_rt_hi = nullptr;
    TRY(a.upload(&d_ct_inst, ct_inst)); TRY(a.upload(&d_ct_lo, ct_lo)); TRY(a.upload(&d_ct_hi, ct_hi));
    if (!rt_inst.empty()) {
      TRY(a.upload(&d_rt_inst, rt_inst)); TRY(a.upload(&d_rt_lo, rt_lo)); TRY(a.upload(&d_rt_hi, rt_hi));
    }
    G.nct = (int32_t)ct_inst.size(); G.ct_inst = d_ct_inst; G.ct_lo = d_ct_lo; G.ct_hi = d_ct_hi;
    G.nrt = (int32_t)rt_inst.size(); G.rt_inst = d_rt_inst; G.rt_lo = d_rt_lo; G.rt_hi = d_rt_hi;
    G.nnz_a = nnz_a; G.nnz_p = nnz_p;
    G.vq_p = nnz_p > 0 ? (nnz_p / n >= 384 ? 4 : nnz_p / n >= 128 ? 2 : 1) : 0;
    if (sizeof(T) == 8) G.vq_p = std::min(G.vq_p, 2);
    grid = std::max(G.nct, G.nrt) * cs;
    // CTAs of each instance's clusters (tiles are per cluster, CS CTAs each)
    std::vector<int32_t> cc_lo(ninst), cc_hi(ninst), cr_lo(ninst), cr_hi(ninst);
    for (int i = 0; i < ninst; ++i) {
      cc_lo[i] = it_lo[i] * cs; cc_hi[i] = it_hi[i] * cs;
      cr_lo[i] = irt_lo[i] * cs; cr_hi[i] = irt_hi[i] * cs;
    }

    // workspace; z and t are padded to whole 16-byte groups and zeroed once
    // (the stage copies read the padding)
    T *dinv, *r, *z, *p, *sv, *t;
    TRY(a.alloc(&dinv, n)); TRY(a.alloc(&r, n)); TRY(a.alloc(&p, n)); TRY(a.alloc(&sv, n));
    TRY(a.alloc(&z, n + 2 * E));
    TRY(a.alloc(&t, std::max<int64_t>(m, 1) + 2 * E));
    CU(cudaMemsetAsync(z, 0, sizeof(T) * (n + 2 * E), st));
    CU(cudaMemsetAsync(t, 0, sizeof(T) * (std::max<int64_t>(m, 1) + 2 * E), st));
    double *part_r, *part_d, *part_c;
    TRY(a.alloc(&part_r, grid)); TRY(a.alloc(&part_d, grid)); TRY(a.alloc(&part_c, 4 * (int64_t)grid));
    CU(cudaMemsetAsync(part_r, 0, sizeof(double) * grid, st));
    CU(cudaMemsetAsync(part_d, 0, sizeof(double) * grid, st));
    CU(cudaMemsetAsync(part_c, 0, sizeof(double) * 4 * grid, st));
    int32_t *d_cc_lo, *d_cc_hi, *d_cr_lo, *d_cr_hi;
    TRY(a.upload(&d_cc_lo, cc_lo)); TRY(a.upload(&d_cc_hi, cc_hi));
    TRY(a.upload(&d_cr_lo, cr_lo)); TRY(a.upload(&d_cr_hi, cr_hi));
    TRY(a.alloc(&bar, 4));
    CU(cudaMallocHost(&h_err, sizeof(int32_t)));
    S.dinv = dinv; S.r = r; S.z = z; S.p = p; S.s = sv; S.t = t;
    S.part_r = part_r; S.part_d = part_d; S.part_c = part_c;
    S.cc_lo = d_cc_lo; S.cc_hi = d_cc_hi; S.cr_lo = d_cr_lo; S.cr_hi = d_cr_hi;
    if (p_diag && !pd_dev) {   // no P: zeros
      TRY(a.alloc(&pd_dev, n));
      CU(cudaMemsetAsync(pd_dev, 0, sizeof(T) * n, st));
    }
    S.short_p = short_p; S.p_diag = p_diag; S.pd = pd_dev; S.nslot = nslot; S.c_split = c_split;
    S.RT = (int32_t)std::max<int64_t>(RT, 1); S.CT = (int32_t)std::max<int64_t>(CT, 1);
    S.RTo = (int32_t)std::max<int64_t>((RT + cs - 1) / cs, 1); S.CTo = (int32_t)std::max<int64_t>((CT + cs - 1) / cs, 1);
    S.sm = sm;
    S.wait_limit = 2000000000LL;   // about 1 s at 2 GHz
    CU(cudaStreamSynchronize(st));
    return COSMO_OK;
  }

  static const void* gcs_kernel(int c) {
    switch (c) {
      case 1: return (const void*)k_gcg_stream<T, 1>;
      case 2: return (const void*)k_gcg_stream<T, 2>;
      case 4: return (const void*)k_gcg_stream<T, 4>;
      default: return (const void*)k_gcg_stream<T, 8>;
    }
  }

  cosmo_status solve(double sigma, const void* rho, const void* rhs, void* x, double tol, int32_t maxit,
                     int32_t* iters, cudaStream_t st) override {
    if (!(sigma > 0.0) || !(tol > 0.0) || maxit < 1 || !rho || !rhs || !x)
      return fail(COSMO_E_INVAL, "bad arguments to cosmo_pcg_plan_solve");
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != device) return fail(COSMO_E_INVAL, "the plan belongs to device %d, device %d is current", device, dev);
    k_gcs_precond<T><<<(int)((n * 32 + 255) / 256), 256, 0, st>>>(n, S.LC, P.P_rp, P.P_ci, P.P_v, sigma,
                                                                  (const T*)rho, const_cast<T*>(S.dinv));
    CU(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st));
    GcsArgs<T> A = S;
    A.rhs = (const T*)rhs; A.x = (T*)x; A.rho = (const T*)rho; A.sigma = sigma;
    A.tol = tol; A.maxit = maxit; A.iters = iters;
    A.ts = ts;
    A.ts_iters = kTsIters;
    if (ts) CU(cudaMemsetAsync(ts, 0, sizeof(unsigned long long) * kTsIters * GCS_NSTAMP * grid, st));
    GridBar B{bar, bar + 1, reinterpret_cast<int32_t*>(bar + 2), 2000000000LL};
    // all clusters resident (cooperative), CS CTAs per cluster
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(GCS_NT);
    cfg.dynamicSmemBytes = (size_t)S.sm.total;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = cs; at[1].val.clusterDim.y = 1; at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    switch (cs) {
      case 1: CU(cudaLaunchKernelEx(&cfg, k_gcg_stream<T, 1>, P, G, A, B)); break;
      case 2: CU(cudaLaunchKernelEx(&cfg, k_gcg_stream<T, 2>, P, G, A, B)); break;
      case 4: CU(cudaLaunchKernelEx(&cfg, k_gcg_stream<T, 4>, P, G, A, B)); break;
      default: CU(cudaLaunchKernelEx(&cfg, k_gcg_stream<T, 8>, P, G, A, B)); break;
    }
    g_launches += 2;
    CU(cudaMemcpyAsync(h_err, bar + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (*h_err) return fail(COSMO_E_TIMEOUT, "streamed CG: a wait gave up");
    if (ts) TRY(reduce_timing());
    return COSMO_OK;
  }

  cosmo_status set_timing(int enable) override {
    if (enable && !ts) {
      TRY(a.alloc(&ts, (int64_t)kTsIters * GCS_NSTAMP * grid));
    } else if (!enable) {
      ts = nullptr;   // the buffer stays in the plan's arena until it is destroyed
    }
    return COSMO_OK;
  }

  // phase k spans stamps k -> k + 1 (the last: stamp 9 -> the next
  // iteration's 0); mean over CTAs and over iterations 1 .. the last full
  // one, and the mean over those iterations of the slowest CTA
  cosmo_status reduce_timing() {
    std::vector<unsigned long long> h((size_t)kTsIters * GCS_NSTAMP * grid);
    CU(cudaMemcpy(h.data(), ts, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    auto at = [&](int it, int k, int b) { return h[((size_t)it * GCS_NSTAMP + k) * grid + b]; };
    for (int ph = 0; ph < COSMO_PCG_PHASES; ++ph) {
      double sum = 0.0, smax = 0.0;
      int cnt = 0;
      for (int it = 1; it + 1 < kTsIters; ++it) {
        double s1 = 0.0, mx = 0.0;
        int nb = 0;
        for (int b = 0; b < grid; ++b) {
          const unsigned long long t0 = at(it, ph, b);
          const unsigned long long t1 = ph + 1 < GCS_NSTAMP ? at(it, ph + 1, b) : at(it + 1, 0, b);
          if (!t0 || !t1 || t1 < t0) continue;
          s1 += (double)(t1 - t0);
          mx = std::max(mx, (double)(t1 - t0));
          ++nb;
        }
        if (nb == grid) {
          sum += s1 / nb;
          smax += mx;
          ++cnt;
        }
      }
      ph_mean[ph] = cnt ? sum / cnt * 1e-3 : 0.0;
      ph_max[ph] = cnt ? smax / cnt * 1e-3 : 0.0;
    }
    return COSMO_OK;
  }

  void get_timing(double* mean_us, double* slowest_us) const override {
    for (int ph = 0; ph < COSMO_PCG_PHASES; ++ph) {
      if (mean_us) mean_us[ph] = ph_mean[ph];
      if (slowest_us) slowest_us[ph] = ph_max[ph];
    }
  }

  void info(cosmo_pcg_plan_info* o) const override {
    o->nseg_a = S.LR.nseg;
    o->nseg_at = S.LC.nseg;
    o->cluster = cs;
    o->ring_slots = nslot;
    o->grid = grid;
    o->threads = GCS_NT;
    o->layout_bytes = layout_bytes;
    o->smem_bytes = S.sm.total;
    o->quads_a = quads_r;
    o->quads_at = quads_c;
  }
};

struct cosmo_pcg_plan {
  std::unique_ptr<PcgPlanBase> impl;
};

static cosmo_status pcg_plan_build(int32_t precision, int32_t ninst, int64_t n, int64_t m, const int64_t* col_off,
                                   const int64_t* row_off, const int64_t* A_rp, const int32_t* A_ci,
                                   const void* A_v, const int64_t* AT_rp, const int32_t* AT_ci, const void* AT_v,
                                   const int64_t* P_rp, const int32_t* P_ci, const void* P_v,
                                   std::unique_ptr<PcgPlanBase>& out, cudaStream_t st) {
  if (ninst < 1 || n < 1 || m < 0 || !col_off || !row_off || !A_rp || !AT_rp ||
      (m > 0 && (!A_ci || !A_v || !AT_ci || !AT_v)) || ((P_rp != nullptr) != (P_ci != nullptr)) ||
      ((P_rp != nullptr) != (P_v != nullptr)))
    return fail(COSMO_E_INVAL, "bad arguments to cosmo_pcg_plan_create");
  auto make = [&](auto tag) -> cosmo_status {
    using T = decltype(tag);
    std::unique_ptr<GcsPlan<T>> pl(new GcsPlan<T>());
    TRY(pl->build(ninst, n, m, col_off, row_off, A_rp, A_ci, (const T*)A_v, AT_rp, AT_ci, (const T*)AT_v, P_rp,
                  P_ci, (const T*)P_v, st));
    out = std::move(pl);
    return COSMO_OK;
  };
  if (precision == COSMO_PREC_FP64) return make(double(0));
  if (precision == COSMO_PREC_MIXED) return make(float(0));
  return fail(COSMO_E_INVAL, "unknown precision");
}

extern "C" {

cosmo_status cosmo_pcg_solve(int32_t precision, int32_t ninst, int64_t n, int64_t m,
                             const int64_t* col_off, const int64_t* row_off,
                             const int64_t* A_rowptr, const int32_t* A_col, const void* A_val,
                             const int64_t* AT_rowptr, const int32_t* AT_col, const void* AT_val,
                             const int64_t* P_rowptr, const int32_t* P_col, const void* P_val,
                             double sigma, const void* rho, const void* rhs, void* x,
                             int32_t warm_start, double tol, int32_t max_iter, int32_t* iters,
                             void* stream) {
  g_err.clear();
  if (ninst < 1 || n < 1 || m < 0 || !col_off || !row_off || !AT_rowptr || !A_rowptr || !rho ||
      !rhs || !x || !(sigma > 0.0) || !(tol > 0.0) || max_iter < 1 ||
      (m > 0 && (!A_col || !A_val || !AT_col || !AT_val)) ||
      ((P_rowptr != nullptr) != (P_col != nullptr)) || ((P_rowptr != nullptr) != (P_val != nullptr)))
    return fail(COSMO_E_INVAL, "bad arguments to cosmo_pcg_solve");
  cudaStream_t st = (cudaStream_t)stream;
  // large zero-start solves (few instances, more than 1e5 nonzeros of A per
  // instance on average) take the grid-wide CG; the rest one CTA per instance
  int64_t nnzA = 0;
  if (m > 0) {
    CU(cudaMemcpyAsync(&nnzA, A_rowptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
  }
  const bool grid = !warm_start && ninst < 148 && nnzA / ninst > 100000;
  if (grid) {
    if (precision == COSMO_PREC_FP64 || precision == COSMO_PREC_MIXED) {
      std::unique_ptr<PcgPlanBase> plan;
      const cosmo_status ps = pcg_plan_build(precision, ninst, n, m, col_off, row_off, A_rowptr, A_col, A_val,
                                             AT_rowptr, AT_col, AT_val, P_rowptr, P_col, P_val, plan, st);
      if (ps == COSMO_OK) return plan->solve(sigma, rho, rhs, x, tol, max_iter, iters, st);
      if (ps != COSMO_E_INVAL) return ps;
      g_err.clear();   // not applicable: the global-memory path below
      auto make = [&](auto tag) {
        using T = decltype(tag);
        Prob<T, T> P{};
        P.ninst = ninst; P.n_total = n; P.m_total = m; P.col_off = col_off; P.row_off = row_off;
        P.A_rp = A_rowptr; P.A_ci = A_col; P.A_v = (const T*)A_val;
        P.AT_rp = AT_rowptr; P.AT_ci = AT_col; P.AT_v = (const T*)AT_val;
        P.P_rp = P_rowptr; P.P_ci = P_col; P.P_v = (const T*)P_val;
        return pcg_solve_grid_t<T>(ninst, n, m, col_off, row_off, P, sigma, rho, rhs, x, tol,
                                   max_iter, iters, st);
      };
      return precision == COSMO_PREC_FP64 ? make(double(0)) : make(float(0));
    }
    return fail(COSMO_E_INVAL, "unknown precision");
  }
  if (precision == COSMO_PREC_FP64)
    return pcg_solve_t<double>(ninst, n, m, col_off, row_off, A_rowptr, A_col, A_val, AT_rowptr,
                               AT_col, AT_val, P_rowptr, P_col, P_val, sigma, rho, rhs, x,
                               warm_start, tol, max_iter, iters, st);
  if (precision == COSMO_PREC_MIXED)
    return pcg_solve_t<float>(ninst, n, m, col_off, row_off, A_rowptr, A_col, A_val, AT_rowptr,
                              AT_col, AT_val, P_rowptr, P_col, P_val, sigma, rho, rhs, x,
                              warm_start, tol, max_iter, iters, st);
  return fail(COSMO_E_INVAL, "unknown precision");
}

cosmo_status cosmo_pcg_plan_create(int32_t precision, int32_t ninst, int64_t n, int64_t m,
                                   const int64_t* col_off, const int64_t* row_off,
                                   const int64_t* A_rowptr, const int32_t* A_col, const void* A_val,
                                   const int64_t* AT_rowptr, const int32_t* AT_col,
                                   const void* AT_val, const int64_t* P_rowptr,
                                   const int32_t* P_col, const void* P_val, cosmo_pcg_plan** out,
                                   void* stream) {
  g_err.clear();
  if (!out) return fail(COSMO_E_INVAL, "out is NULL");
  *out = nullptr;
  std::unique_ptr<cosmo_pcg_plan> pl(new cosmo_pcg_plan());
  TRY(pcg_plan_build(precision, ninst, n, m, col_off, row_off, A_rowptr, A_col, A_val, AT_rowptr, AT_col,
                     AT_val, P_rowptr, P_col, P_val, pl->impl, (cudaStream_t)stream));
  *out = pl.release();
  return COSMO_OK;
}

cosmo_status cosmo_pcg_plan_solve(cosmo_pcg_plan* plan, double sigma, const void* rho,
                                  const void* rhs, void* x, double tol, int32_t max_iter,
                                  int32_t* iters, void* stream) {
  g_err.clear();
  if (!plan || !plan->impl) return fail(COSMO_E_INVAL, "plan is NULL");
  return plan->impl->solve(sigma, rho, rhs, x, tol, max_iter, iters, (cudaStream_t)stream);
}

cosmo_status cosmo_pcg_plan_get_info(const cosmo_pcg_plan* plan, cosmo_pcg_plan_info* out) {
  g_err.clear();
  if (!plan || !plan->impl || !out) return fail(COSMO_E_INVAL, "plan or out is NULL");
  plan->impl->info(out);
  return COSMO_OK;
}

cosmo_status cosmo_pcg_plan_set_timing(cosmo_pcg_plan* plan, int32_t enable) {
  g_err.clear();
  if (!plan || !plan->impl) return fail(COSMO_E_INVAL, "plan is NULL");
  return plan->impl->set_timing(enable);
}

cosmo_status cosmo_pcg_plan_get_timing(const cosmo_pcg_plan* plan, double* mean_us, double* slowest_us) {
  g_err.clear();
  if (!plan || !plan->impl) return fail(COSMO_E_INVAL, "plan is NULL");
  plan->impl->get_timing(mean_us, slowest_us);
  return COSMO_OK;
}

cosmo_status cosmo_pcg_plan_destroy(cosmo_pcg_plan* plan) {
  g_err.clear();
  delete plan;
  return COSMO_OK;
}

cosmo_status cosmo_psd_project(int32_t precision, int32_t nblk, const int32_t* p_host,
                               const int64_t* off_host, const void* v, void* out, void* lam,
                               void* U, void* stream) {
  g_err.clear();
  if (nblk < 0 || (nblk > 0 && (!p_host || !off_host || !v || !out)))
    return fail(COSMO_E_INVAL, "bad arguments to cosmo_psd_project");
  if (nblk == 0) return COSMO_OK;
  if (precision == COSMO_PREC_FP64)
    return psd_project_t<double>(nblk, p_host, off_host, v, out, lam, U, (cudaStream_t)stream);
  if (precision == COSMO_PREC_MIXED)
    return psd_project_t<float>(nblk, p_host, off_host, v, out, lam, U, (cudaStream_t)stream);
  return fail(COSMO_E_INVAL, "unknown precision");
}

cosmo_status cosmo_psd_dk_backward(int32_t precision, int32_t nblk, const int32_t* p_host,
                                   const int64_t* off_host, const void* lam, const void* U,
                                   const void* g, void* out, double tau, void* stream) {
  g_err.clear();
  if (nblk < 0 || (nblk > 0 && (!p_host || !off_host || !lam || !U || !g || !out)))
    return fail(COSMO_E_INVAL, "bad arguments to cosmo_psd_dk_backward");
  if (nblk == 0) return COSMO_OK;
  if (precision == COSMO_PREC_FP64)
    return psd_dk_t<double>(nblk, p_host, off_host, lam, U, g, out, tau, (cudaStream_t)stream);
  if (precision == COSMO_PREC_MIXED)
    return psd_dk_t<float>(nblk, p_host, off_host, lam, U, g, out, tau, (cudaStream_t)stream);
  return fail(COSMO_E_INVAL, "unknown precision");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of the standalone reduced-system solve.
//
// Some callers cannot allocate device memory once they are running: a
// fixed-rate control loop (an MPC or covariance-steering controller that
// calls the solver every few milliseconds) cannot afford cudaMalloc's latency,
// its implicit device synchronisation or the chance that it fails mid-run;
// hosts that hand the library a fixed device budget up front may forbid any
// allocation outside it.  For them the CG workspace lives in one file-scope
// device array, reserved when the library is loaded and held on every GPU that
// loads it until the process exits.
//
// Host code may not pass g_pcg_scratch itself to a kernel: on the host that
// name is only a stand-in for the device symbol.  The first call in each CUDA
// context looks up the symbol's device address (cudaGetSymbolAddress, with
// that context's device current) and caches it per context; that first call
// should therefore happen before any stream capture.  Every call shares the one array, so calls that
// overlap on the GPU (different streams, or different host threads on the
// same device) race on it; the caller must order them.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_pcg_scratch[COSMO_PCG_NOALLOC_MAX_BYTES];

static std::mutex g_scratch_mu;
// (context, device address) of the array, one entry per driver context that
// has called: a context created after cudaDeviceReset, or a non-primary
// context made current by the caller, gets its own lookup instead of a stale
// address.  The context handle comes from the driver's cuCtxGetCurrent,
// reached through the runtime's entry-point query (no link against libcuda).
struct ScratchEntry { void* ctx; void* addr; };
static ScratchEntry g_scratch_cache[64];
static int g_scratch_n = 0;

// the calling thread's current driver context (null when the runtime has not
// made one current yet)
static cosmo_status current_context(void** ctx) {
  typedef int (*CtxGetCurrentFn)(void**);
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f) {
      cudaGetLastError();
      return fail(COSMO_E_CUDA, "driver entry point cuCtxGetCurrent unavailable");
    }
    fn = reinterpret_cast<CtxGetCurrentFn>(f);
  }
  *ctx = nullptr;
  if (fn(ctx) != 0) return fail(COSMO_E_CUDA, "cuCtxGetCurrent failed");
  return COSMO_OK;
}

static cosmo_status scratch_address(void** out) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  void* ctx = nullptr;
  TRY(current_context(&ctx));
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (ctx)
    for (int i = 0; i < g_scratch_n && i < 64; ++i)
      if (g_scratch_cache[i].ctx == ctx) { *out = g_scratch_cache[i].addr; return COSMO_OK; }
  // the lookup also makes the device's primary context current if none was
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_pcg_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return fail(COSMO_E_CUDA, "cudaGetSymbolAddress of the solve scratch failed on device %d: %s",
                dev, cudaGetErrorString(e));
  }
  if (!ctx) TRY(current_context(&ctx));
  if (ctx) g_scratch_cache[g_scratch_n++ % 64] = ScratchEntry{ctx, p};   // a full table reuses its oldest slot
  *out = p;
  return COSMO_OK;
}

template <class T>
static cosmo_status pcg_solve_noalloc_t(int32_t ninst, int64_t n, int64_t m, const int64_t* col_off,
                                        const int64_t* row_off, const int64_t* A_rp,
                                        const int32_t* A_ci, const void* A_v, const int64_t* AT_rp,
                                        const int32_t* AT_ci, const void* AT_v, const int64_t* P_rp,
                                        const int32_t* P_ci, const void* P_v, double sigma,
                                        const void* rho, const void* rhs, void* x, int32_t warm,
                                        double tol, int32_t maxit, int32_t* iters,
                                        cudaStream_t st) {
  const size_t need = sizeof(T) * (size_t)(4 * n + m) + sizeof(int32_t) * 2 * (size_t)ninst;
  if (need > (size_t)COSMO_PCG_NOALLOC_MAX_BYTES)
    return fail(COSMO_E_INVAL,
                "cosmo_pcg_solve_noalloc: n=%lld, m=%lld, ninst=%d need %zu bytes of scratch, "
                "above the fixed maximum of %d bytes",
                (long long)n, (long long)m, ninst, need, (int)COSMO_PCG_NOALLOC_MAX_BYTES);
  void* base = nullptr;
  TRY(scratch_address(&base));
  T* dinv = reinterpret_cast<T*>(base);
  T* r = dinv + n;
  T* p = r + n;
  T* u = p + n;
  T* t = u + n;
  int32_t* flags = reinterpret_cast<int32_t*>(t + m);
  int32_t* sched = flags + ninst;
  Prob<T, T> P{};
  P.ninst = ninst; P.n_total = n; P.m_total = m; P.col_off = col_off; P.row_off = row_off;
  P.A_rp = A_rp; P.A_ci = A_ci; P.A_v = (const T*)A_v;
  P.AT_rp = AT_rp; P.AT_ci = AT_ci; P.AT_v = (const T*)AT_v;
  P.P_rp = P_rp; P.P_ci = P_ci; P.P_v = (const T*)P_v;
  P.inst_sched = sched;
  // the array keeps the previous call's contents: the flag words must start at zero
  CU(cudaMemsetAsync(flags, 0, sizeof(int32_t) * ninst, st));
  k_iota<<<grid_for(ninst, 256), 256, 0, st>>>(ninst, sched);
  k_precond_csr<T, T><<<grid_for(n, 256), 256, 0, st>>>(P, sigma, (const T*)rho, dinv);
  CgArgs<T> ca{};
  ca.rhs = (const T*)rhs; ca.x = (T*)x; ca.x0 = nullptr; ca.rho = (const T*)rho; ca.dinv = dinv;
  ca.sigma = sigma; ca.r = r; ca.p = p; ca.u = u; ca.t = t; ca.tol = tol; ca.maxit = maxit;
  ca.zero_start = warm ? 0 : 1; ca.flag_bit = F_CG_CAP; ca.flags = flags; ca.iters = iters;
  k_pcg<T, T, 256><<<ninst, 256, 0, st>>>(P, ca);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(COSMO_E_CUDA, "pcg launch failed: %s", cudaGetErrorString(e));
  g_launches += 3;
  return COSMO_OK;
}

extern "C" cosmo_status cosmo_pcg_solve_noalloc(
    int32_t precision, int32_t ninst, int64_t n, int64_t m, const int64_t* col_off,
    const int64_t* row_off, const int64_t* A_rowptr, const int32_t* A_col, const void* A_val,
    const int64_t* AT_rowptr, const int32_t* AT_col, const void* AT_val, const int64_t* P_rowptr,
    const int32_t* P_col, const void* P_val, double sigma, const void* rho, const void* rhs,
    void* x, int32_t warm_start, double tol, int32_t max_iter, int32_t* iters, void* stream) {
  g_err.clear();
  if (ninst < 1 || n < 1 || m < 0 || !col_off || !row_off || !AT_rowptr || !A_rowptr || !rho ||
      !rhs || !x || !(sigma > 0.0) || !(tol > 0.0) || max_iter < 1 ||
      (m > 0 && (!A_col || !A_val || !AT_col || !AT_val)) ||
      ((P_rowptr != nullptr) != (P_col != nullptr)) || ((P_rowptr != nullptr) != (P_val != nullptr)))
    return fail(COSMO_E_INVAL, "bad arguments to cosmo_pcg_solve_noalloc");
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == COSMO_PREC_FP64)
    return pcg_solve_noalloc_t<double>(ninst, n, m, col_off, row_off, A_rowptr, A_col, A_val,
                                       AT_rowptr, AT_col, AT_val, P_rowptr, P_col, P_val, sigma,
                                       rho, rhs, x, warm_start, tol, max_iter, iters, st);
  if (precision == COSMO_PREC_MIXED)
    return pcg_solve_noalloc_t<float>(ninst, n, m, col_off, row_off, A_rowptr, A_col, A_val,
                                      AT_rowptr, AT_col, AT_val, P_rowptr, P_col, P_val, sigma,
                                      rho, rhs, x, warm_start, tol, max_iter, iters, st);
  return fail(COSMO_E_INVAL, "unknown precision");
}
