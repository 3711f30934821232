/*
 * cosmo_du.h -- C ABI of the B300 (sm_103a) library for one unrolled COSMO
 * ADMM iteration and its backward, batched over many conic programs.
 *
 * Problem (Sec. 2.1, Eq. conic-standard), one per instance i:
 *     minimize 1/2 x'Px + q'x   s.t.  A x + s = b,  s in K
 * K is a product of zero, nonnegative, box, second-order (SOC) and PSD cones
 * listed in row order.  PSD blocks are stored in svec form: upper triangle,
 * column by column, off-diagonals times sqrt(2) (an isometry, so projections
 * and their adjoints need no extra factors).
 *
 * Iteration k (Sec. 2.2, Eqs. cosmo_linear_system .. cosmo_projection) with
 * per-row penalties rho^k (rectified to the block mean on SOC/PSD blocks,
 * App. E), relaxation alpha^k per instance and sigma_k:
 *     (P + sigma I + A'D(rho)A) x~ = sigma x - q + A'(y + rho o (b - s))   (Sec. 2.3, reduced form)
 *     s~ = b - A x~                         (equal to s - (y + nu~)/rho)
 *     x+ = alpha x~ + (1 - alpha) x
 *     s+ = Pi_K(alpha s~ + (1 - alpha) s + y / rho)
 *     y+ = y + rho o (alpha s~ + (1 - alpha) s - s+)
 * The linear system is solved matrix-free by Jacobi-preconditioned CG (App. D),
 * warm-started at the previous x~.  The backward uses the adjoint CG rule of
 * Sec. 2.3 (Eq. grad_rho) and the Daleckii-Krein rule of Sec. 2.4
 * (Eqs. psd-cotangent-dk, lowner).
 *
 * Conventions
 *  - Every function returns a cosmo_status; no C++ exception crosses the ABI.
 *    On failure cosmo_last_error() returns a thread-local message.
 *  - "dev" pointers are caller-owned device memory (e.g. PyTorch tensors),
 *    "host" pointers caller-owned host memory.  The library never frees
 *    caller memory; it owns only the opaque batch and what the batch
 *    allocates (problem copy, tape, workspace).
 *  - Real-valued device arrays ("real") are float for COSMO_PREC_MIXED and
 *    double for COSMO_PREC_FP64.  Reductions (norms, losses, CG inner
 *    products, eigenvalue-gap tests) are done in double in both modes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered and do not synchronise unless the
 *    name says so (cosmo_status_sync, cosmo_step_host).
 *  - Batched arrays concatenate instances: x, q have n_total entries, s, y,
 *    b have m_total; instance i owns the column range [col_off[i],
 *    col_off[i+1]) and the row range [row_off[i], row_off[i+1]).
 *  - Conditions found on the device (CG cap reached, non-finite values,
 *    eigensolver sweep cap, invalid rho/alpha) set per-instance flag bits
 *    read by cosmo_status_sync; they never trap.
 */
#ifndef COSMO_DU_H
#define COSMO_DU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  COSMO_OK = 0,
  COSMO_E_INVAL = 1,      /* invalid argument or problem data */
  COSMO_E_NOMEM = 2,      /* device or host allocation failed */
  COSMO_E_CUDA = 3,       /* a CUDA runtime call failed */
  COSMO_E_NOTCONV = 4,    /* (flag) CG reached its iteration cap */
  COSMO_E_NONFINITE = 5,  /* (flag) a non-finite iterate was produced */
  COSMO_E_TIMEOUT = 6,    /* a bounded device wait gave up (grid-wide CG barrier) */
  COSMO_E_STATE = 7,      /* call out of order (e.g. backward without tape) */
  COSMO_E_NODEVICE = 8    /* no CUDA device */
} cosmo_status;

/* cone types (Sec. 2.4 lists zero, orthant, SOC, PSD; box is an addition) */
enum {
  COSMO_CONE_ZERO = 0,
  COSMO_CONE_NONNEG = 1,
  COSMO_CONE_BOX = 2,
  COSMO_CONE_SOC = 3,
  COSMO_CONE_PSD = 4
};

/* precision modes */
enum {
  COSMO_PREC_MIXED = 0, /* float iterates and values, double reductions */
  COSMO_PREC_FP64 = 1   /* double everywhere */
};

/* storage of the matrix values of P and A in COSMO_PREC_MIXED */
enum { COSMO_VAL_F32 = 0, COSMO_VAL_BF16 = 1 };

/* per-instance flag bits reported by cosmo_status_sync */
enum {
  COSMO_FLAG_CG_CAP = 1,        /* forward CG hit cg_max_iter */
  COSMO_FLAG_ADJ_CG_CAP = 2,    /* adjoint CG hit cg_max_iter */
  COSMO_FLAG_EIG_CAP = 4,       /* eigensolver hit its sweep/iteration cap */
  COSMO_FLAG_NONFINITE = 8,     /* non-finite iterate or cotangent */
  COSMO_FLAG_BAD_PARAM = 16,    /* rho <= 0, non-finite, or alpha outside (0, 2) */
  COSMO_FLAG_TIMEOUT = 32       /* a bounded device wait gave up (tensor-core DK backward) */
};

/* One cone: type and dimension.  For PSD, dim = p and the cone occupies
 * p(p+1)/2 rows; for every other type it occupies dim rows. */
typedef struct {
  int32_t type;
  int32_t dim;
} cosmo_cone;

/* Problem batch, all HOST memory, read during cosmo_batch_create only
 * (the library copies what it needs).  CSR arrays are batch-global: rows of
 * A are the concatenated constraint rows, columns are global variable
 * indices; every row of instance i must only reference columns of instance i
 * (the batch is block diagonal).  P holds both triangles of each symmetric
 * block; P_rowptr may be NULL for P = 0. */
typedef struct {
  int32_t ninst;
  const int64_t* col_off;   /* [ninst+1], col_off[0] = 0, nondecreasing */
  const int64_t* row_off;   /* [ninst+1] */
  const int64_t* P_rowptr;  /* [n_total+1] or NULL */
  const int32_t* P_col;     /* [nnzP] */
  const double* P_val;      /* [nnzP] */
  const int64_t* A_rowptr;  /* [m_total+1] */
  const int32_t* A_col;     /* [nnzA] */
  const double* A_val;      /* [nnzA] */
  const double* q;          /* [n_total] */
  const double* b;          /* [m_total] */
  const double* box_l;      /* [m_total] or NULL (required if a box cone exists) */
  const double* box_u;      /* [m_total] or NULL */
  const int32_t* cone_count;/* [ninst] cones of each instance */
  const cosmo_cone* cones;  /* [sum cone_count], instance by instance, row order */
} cosmo_problem;

typedef struct {
  int32_t precision;        /* COSMO_PREC_MIXED or COSMO_PREC_FP64 */
  int32_t value_type;       /* COSMO_VAL_F32 / COSMO_VAL_BF16 (MIXED only): storage of A
                               and A'.  P is stored in the iterate type: entrywise BF16
                               rounding of P = M'M + reg I perturbs it by more than its
                               smallest eigenvalue and can make the QP nonconvex. */
  double cg_tol;            /* stop when ||r|| <= cg_tol * ||rhs|| (App. D: 1e-8) */
  int32_t cg_max_iter;      /* CG cap per solve; flag COSMO_FLAG_*CG_CAP */
  int32_t checkpoint_every; /* 0: keep the whole tape; c > 0: keep states every
                               c steps and recompute segments in the backward */
  double dk_gap_tau;        /* Loewner-matrix gap threshold, relative:
                               tau = dk_gap_tau * max(1, max|lambda|) */
  int32_t eig_jacobi_max_p; /* PSD blocks with p <= this use the cyclic Jacobi
                               solver (shared memory), larger ones Householder
                               tridiagonalisation + implicit QL (global memory)
                               and a global-memory DK backward; <= 0: every
                               block whose warm-started Jacobi fits in shared
                               memory uses Jacobi */
  int32_t eig_max_sweeps;   /* Jacobi sweep cap (flag COSMO_FLAG_EIG_CAP) */
  double eig_tol;           /* Jacobi stop: off(A) <= eig_tol * ||A||_F */
  int32_t use_graph;        /* capture forward/backward into CUDA graphs */
  int32_t device;           /* CUDA device ordinal the batch lives on */
  int32_t eig_warm_start;   /* 1: start step k's Jacobi from step k-1's eigenvectors
                               (re-orthogonalised by one Newton-Schulz step) */
  int32_t dk_tensor_cores;  /* 1: MIXED-precision DK backward of blocks of order <= 80 on
                               the tensor cores (tcgen05, split-TF32 products); 0: CUDA cores */
  int32_t cg_cluster;       /* CTAs per instance in the CG: 0 automatic (1 with the
                               instance's vectors in shared memory when 5 n_i + m_i reals
                               fit in 200 KB; else 2 or 4 for fewer than 74 / 37 instances
                               with >= 8192 rows + columns, else 1); 1 (shared-memory
                               vectors when they fit), 2 or 4 forced; one CTA per instance
                               forced: -1 vectors in shared memory, -2 vectors and the
                               instance's A, A' and P in shared memory, -3 global-memory
                               vectors (-1 / -2 fail with E_INVAL at creation when the
                               data does not fit in 200 KB); -4 one warp per instance
                               over global vectors (offered to the autotuner when every
                               CG instance has n_i + m_i <= 4096 and nnz(A_i) + nnz(P_i)
                               <= 16384; measured slower than -2 on the covariance-
                               steering instances, so never the shape rules' choice) */
  int32_t loss_kind;        /* per-instance loss of cosmo_forward / cotangent of
                               cosmo_backward: 0 ||r_p^K||^2 + ||r_d^K||^2; 1 the log-residual
                               loss of Sec. 4, sum_{k=1..K} log(||r_d^k||^2/||r_d^0||^2 +
                               ||r_p^k||^2/||r_p^0||^2), k = 0 norms held constant, a term with
                               a zero k = 0 norm dropped */
  int32_t eig_variant;      /* Jacobi kernel of the PSD projection: 0 automatic (3 where it
                               has an instantiation for the class and CTA size, else 2), 1 the
                               matrix and eigenvectors by index (two barriers per round),
                               2 the matrix in round-robin slot order as 2x2 tiles with the
                               next round's rotations formed in the same pass (one barrier
                               per round), 3 the same solver on a compile-time geometry per
                               size class (orders up to 8, 16, 32, 56, 80; eigenvectors kept by slot
                               in a double buffer; a class without an instantiation for its
                               CTA size is an error).  All give the eigen-decomposition to
                               eig_tol. */
  int32_t eig_threads;      /* CTA size of the Jacobi projection: 0 by block order (64 up
                               to p = 16 on the compile-time geometry, 128 up to 32, 256 up
                               to 56, 512 above), or 128, 256, 512 (or
                               1024 with eig_variant 0, 2 or 3) for every block */
  int32_t autotune;         /* 1: at batch creation, time the candidate launch
                               configurations of what the options leave automatic and keep
                               the fastest (see cosmo_tuning); 0: shape rules only */
  int32_t fwd_persistent;   /* 1: in MIXED precision with FP32 values, where every instance
                               has a diagonal reduced system and exactly one PSD block (its
                               other rows zero, nonnegative or box; no SOC) and every size
                               class runs the compile-time-geometry Jacobi, one launch per
                               size class runs all steps of a forward segment (one CTA per
                               instance: a3..a8 step after step, no per-step launches; the
                               open-loop forward with loss_kind 0 only); results equal the
                               per-step launches bit for bit.  0 (default): per-step
                               launches (measured faster on the batched max-cut workload
                               in graph mode: 13.0 against 15.0 ms per forward). */
} cosmo_options;

/* Launch configuration of a batch: the PSD size classes (blocks sorted by
 * order, largest first, split where the CTA-size rule changes) with the
 * eigensolver and CTA size of each, and the CG kernel.  Filled by the shape
 * rules, or by the autotuner (option autotune = 1), which at batch creation
 * times on the device, with synthetic data of the batch's own shapes:
 *   - per class, the slot-layout Jacobi at CTA sizes 128 / 256 / 512 / 1024
 *     and, on the compile-time geometry of orders above 32, 384 (those that
 *     fit, each on the compile-time geometry where it has an instantiation; projection of a perturbed block warm-started from the
 *     eigenvectors of the unperturbed one), and for classes of order >= 48
 *     the tridiagonal + QL path, each with its backward (Daleckii-Krein)
 *     kernel;
 *   - the CG kernel: one CTA per instance with the instance's data in shared
 *     memory (-2), its vectors in shared memory (-1), global vectors (-3),
 *     or clusters of 2 / 4 CTAs (20 iterations of the batch's operator);
 * keeping the fastest.  A choice is cached per process for the same device,
 * precision and shapes.  Only what the options leave automatic is tuned
 * (eig_threads 0, eig_variant 0, 2 or 3, eig_jacobi_max_p 0, cg_cluster 0). */
#define COSMO_MAX_PSD_CLASSES 8
typedef struct {
  int32_t n_classes;
  int32_t class_maxp[COSMO_MAX_PSD_CLASSES];     /* largest order of the class */
  int32_t class_count[COSMO_MAX_PSD_CLASSES];    /* blocks in the class */
  int32_t class_method[COSMO_MAX_PSD_CLASSES];   /* 0 Jacobi in shared memory (eig_variant),
                                                    1 tridiagonal + implicit QL,
                                                    2 one block per thread (MIXED, orders
                                                    <= 8: serial cyclic Jacobi with the same
                                                    refinement, CUDA-core DK backward); the
                                                    shape rules choose 2 for such classes
                                                    when eig_variant and eig_threads are 0 */
  int32_t class_threads[COSMO_MAX_PSD_CLASSES];  /* CTA size of the projection */
  int32_t cg_kernel;        /* 0 the shape rule (or no CG), else a cg_cluster value */
  int32_t tuned;            /* 1 if the autotuner chose this configuration */
  double tune_ms;           /* host time spent tuning at creation (0 if cached or off) */
} cosmo_tuning;

typedef struct {
  int32_t ninst;
  int32_t precision;
  int64_t n_total, m_total;
  int64_t nnzA, nnzP;
  int32_t n_soc, n_psd, max_psd_p;
  int64_t psd_u_entries;    /* sum of p^2 over PSD blocks */
  int64_t device_bytes;     /* device memory the batch currently owns */
  int32_t last_K;           /* K of the last forward (0 if none) */
  int32_t tape_valid;       /* 1 if a backward can run now */
  int64_t kernels_launched; /* kernels this batch launched so far (graph replays
                               count their kernels) */
  /* work counters since creation (cosmo_batch_get_info synchronises to read them) */
  int64_t eig_sweeps, eig_blocks;       /* Jacobi sweeps summed over PSD-block projections */
  int64_t cg_iters, cg_solves;          /* forward CG iterations / solves (per instance) */
  int64_t adj_cg_iters, adj_cg_solves;  /* adjoint CG iterations / solves */
  int32_t fwd_persistent;   /* 1 if the batch's forward runs persistent (option
                               fwd_persistent and the batch qualifies), else 0 */
} cosmo_batch_info;

typedef struct cosmo_batch cosmo_batch;

/* Library version and the number of kernels launched by all batches. */
const char* cosmo_version(void);
int64_t cosmo_kernel_launch_count(void);

/* Thread-local message of the last failing call ("" if none). */
const char* cosmo_last_error(void);

/* Fill *opt with defaults for a precision mode: MIXED cg_tol 1e-8, FP64 1e-10;
 * cg_max_iter 500; checkpoint_every 0; dk_gap_tau 1e-12; eig_jacobi_max_p 0
 * (Jacobi wherever it fits in shared memory); 30 sweeps; eig_tol 1e-6 (MIXED) / 1e-14 (FP64);
 * use_graph 1; device 0; eig_warm_start 1; dk_tensor_cores 1; cg_cluster 0; loss_kind 0;
 * eig_variant 0; eig_threads 0; autotune 0; fwd_persistent 0.
 * Returns COSMO_E_INVAL for an unknown precision. */
cosmo_status cosmo_options_default(cosmo_options* opt, int32_t precision);

/* The batch's launch configuration (see cosmo_tuning).  Errors: E_INVAL. */
cosmo_status cosmo_batch_get_tuning(const cosmo_batch* b, cosmo_tuning* out);

/* Impose a launch configuration, e.g. one read from another batch of the same
 * shapes: n_classes and class_maxp / class_count must match this batch's
 * classes; every method / CTA size / CG kernel must fit (E_INVAL otherwise,
 * nothing changed).  Recorded CUDA graphs are dropped and captured again.
 * Synchronises the device. */
cosmo_status cosmo_batch_set_tuning(cosmo_batch* b, const cosmo_tuning* t);

/* Validate a problem on the host without touching the device (CSR bounds and
 * block-diagonal structure, cone rows summing to each instance's row count,
 * PSD dims, box bounds l <= u, finite data).  COSMO_OK or COSMO_E_INVAL. */
cosmo_status cosmo_problem_validate(const cosmo_problem* prob);

/* Create a batch on opt->device: validates (as above, before any CUDA call),
 * builds A' in CSR, the cone schedule and the Jacobi-preconditioner
 * ingredients, and uploads them.  *out is owned by the caller and released
 * with cosmo_batch_destroy.  Errors: E_INVAL, E_NODEVICE, E_NOMEM, E_CUDA. */
cosmo_status cosmo_batch_create(const cosmo_problem* prob, const cosmo_options* opt,
                                cosmo_batch** out);
cosmo_status cosmo_batch_destroy(cosmo_batch* batch);
cosmo_status cosmo_batch_get_info(const cosmo_batch* batch, cosmo_batch_info* out);

/* Solve to tolerance: the vanilla COSMO baseline of Sec. 4 (App. D: the
 * unrolled iteration with the OSQP-style residual-balancing rho heuristic,
 * a zero or given start, alpha fixed).  Each instance has one scalar rho_i
 * (rho_eq_scale * rho_i on zero-cone rows); every check_every iterations the
 * KKT residuals are measured in the infinity norm and normalised OSQP-style,
 *   rbar_p = ||Ax + s - b|| / max(||Ax||, ||s||, ||b||),
 *   rbar_d = ||Px + q - A'y|| / max(||Px||, ||q||, ||A'y||)
 * (a zero scale counts as 1; the sign of r_d as in cosmo_residuals).  An
 * instance has converged at the first check with rbar_p <= eps and rbar_d
 * <= eps.  At every rebalance_every-th iteration (a multiple of check_every;
 * 0 keeps rho fixed) an unconverged instance's rho_i is multiplied by
 * f = sqrt(rbar_p / rbar_d) when f > rebalance_tol or f < 1 / rebalance_tol,
 * then clipped to [rho_min, rho_max].  The loop ends when every instance has
 * converged or after max_iter iterations; converged instances keep
 * iterating until then.  The paper leaves the check and rebalancing
 * intervals and the threshold open; cosmo_solve_params_default sets sigma
 * 1e-6, alpha 1.6, rho0 0.1, rho_eq_scale 1e3, eps 1e-3, rebalance_tol 5,
 * rho in [1e-6, 1e6], max_iter 5000, checks and rebalancing every 25
 * iterations.
 * x [n], s [m], y [m]: device, the start in and the final iterate out.
 * iters [ninst] (host, may be NULL): the iteration count of each instance's
 * first converged check, -1 if it never converged.  rbar_p, rbar_d, rho
 * [ninst] (host, may be NULL): the normalised residuals at the last check
 * and the final rho_i.  Runs the forward of the batch (no tape) in chunks of
 * check_every steps, synchronising the stream at every check.
 * Errors: E_INVAL, E_NOMEM, E_CUDA (and those of cosmo_forward). */
typedef struct {
  double sigma, alpha, rho0, rho_eq_scale, eps, rebalance_tol, rho_min, rho_max;
  int32_t max_iter, check_every, rebalance_every, pad;
} cosmo_solve_params;
cosmo_status cosmo_solve_params_default(cosmo_solve_params* p);
cosmo_status cosmo_solve(cosmo_batch* batch, const cosmo_solve_params* prm, void* x, void* s, void* y,
                         int32_t* iters, double* rbar_p, double* rbar_d, double* rho, void* stream);

/* Closed-loop hyperparameter policy of App. E.  Step k of the unrolled
 * iteration uses, per row, rho^k = exp(span sig(l^k_rho) + log 1e-3) (span =
 * log 1e3 - log 1e-3: rho in (1e-3, 1e3)) before the SOC / PSD
 * rectification, and per instance alpha^k = 2 sig(l^k_alpha).  The logits
 * are recurrent, l^{k+1} = l^k + MLP(xi^k), with ReLU MLPs of 32 x 32 hidden
 * units and one output: per row on
 *   xi_rho = [l_rho, s, y, rbar_p, log(||rbar_d||_inf + 1e-12), delta_p, delta_d]
 * and per instance on
 *   xi_alpha = [l_alpha, log(||rbar_p||_inf + 1e-12), log(||rbar_d||_inf +
 *               1e-12), log(||delta_p||_inf + 1e-12), log(||delta_d||_inf + 1e-12)]
 * of the iterate k: rbar_p = (Ax + s - b) / max(||Ax||, ||s||, ||b||) and
 * rbar_d = (Px + q - A'y) / max(||Px||, ||q||, ||A'y||) (infinity norms, a
 * zero scale counts as 1), delta_d = s^k - s^{k-1}, delta_p = s^k - s~^k
 * (s~ before relaxation; both zero at k = 0).  K steps evaluate the policy
 * K - 1 times.  l0 [5] = initial logits (zero rows, orthant and box rows,
 * SOC rows, PSD rows, alpha); the defaults rho = (100, 0.1, 0.1, 0.1) and
 * alpha = 1.6 correspond to logit((log rho + log 1e3) / span) and logit(0.8).
 * Parameter layout of each MLP: W1 [F][32], b1 [32], W2 [32][32], b2 [32],
 * W3 [32][1], b3 [1] (F = 7 and 5; cosmo_policy_sizes: 1345 and 1281).
 * cosmo_policy_forward: as cosmo_forward, with the per-step rho and alpha
 * produced by the policy on the device inside the unrolled sequence (one
 * CUDA graph with use_graph); theta_rho, theta_alpha, l0 are device arrays
 * of the batch's real type, copied at the call.  cosmo_policy_backward: the
 * gradients of <gx, x^K> + <gs, s^K> + <gy, y^K> + sum_i gloss_i loss_i with
 * respect to theta_rho, theta_alpha, l0 (device, same layouts) and, if not
 * NULL, the start (gx0, gs0, gy0), with the features built from the solver
 * state held constant: the gradient reaches the policy through rho^k,
 * alpha^k and the logit recurrence (the l input of each MLP stays live).
 * Parameter sums run in a fixed order.  cosmo_policy_schedule copies the
 * rho [K][m] (before rectification) and alpha [K][ninst] of the last policy
 * forward.  Errors: E_INVAL, E_STATE (backward without a taped policy
 * forward), E_NOMEM, E_CUDA. */
cosmo_status cosmo_policy_sizes(int32_t* n_theta_rho, int32_t* n_theta_alpha);
cosmo_status cosmo_policy_forward(cosmo_batch* batch, int32_t K, const double* sigma_host,
                                  const void* theta_rho, const void* theta_alpha, const void* l0,
                                  const void* x0, const void* s0, const void* y0, void* xK, void* sK,
                                  void* yK, double* loss, int32_t record_tape, void* stream);
cosmo_status cosmo_policy_backward(cosmo_batch* batch, const void* gx, const void* gs, const void* gy,
                                   const double* gloss, void* gtheta_rho, void* gtheta_alpha, void* gl0,
                                   void* gx0, void* gs0, void* gy0, void* stream);
cosmo_status cosmo_policy_schedule(cosmo_batch* batch, void* rho, void* alpha, void* stream);

/* Warm-start network of App. E: two shared ReLU MLPs (two hidden layers of
 * width 64) predict the initial iterate elementwise,
 *   x0_j         = MLP_x([q_j, P_jj, ||A_{:,j}||_2, nnz(A_{:,j}), ctx])
 *   (s0_r, y0_r) = MLP_c([b_r, ||A_{r,:}||_2, nnz(A_{r,:}), onehot5(cone of
 *                         row r: zero, nonneg, box, soc, psd), ctx])
 * with ctx = (log(1 + ||q||_inf), log(1 + ||b||_inf), log(1 + n_i),
 * log(1 + m_i)) of the element's instance.  A layer is h = relu(W' u + b);
 * the output layer is affine.  Parameters of an MLP with F inputs and O
 * outputs, flattened in this order: W1 [F][64], b1 [64], W2 [64][64],
 * b2 [64], W3 [64][O], b3 [O] (F = 8, O = 1 for MLP_x; F = 12, O = 2 for
 * MLP_c); cosmo_ws_sizes gives the two lengths (4801 and 5122).
 * All arrays are device memory of the batch's real type.
 * cosmo_ws_forward: theta_x, theta_c in; x0 [n], s0 [m], y0 [m] out (s0,
 * y0 may be NULL when m = 0).  cosmo_ws_backward: the gradients of
 * <gx0, x0> + <gs0, s0> + <gy0, y0> with respect to theta_x and theta_c,
 * written to gtheta_x, gtheta_c (same layouts); the weight gradients are
 * summed over elements in a fixed order (bitwise reproducible).  The first
 * backward allocates 256 reals per element of max(n, m) for the reverse
 * pass; features are recomputed from the batch on every call.  Both are
 * asynchronous on stream.  Errors: E_INVAL (a NULL operand), E_NOMEM,
 * E_CUDA. */
cosmo_status cosmo_ws_sizes(int32_t* n_theta_x, int32_t* n_theta_c);
cosmo_status cosmo_ws_forward(cosmo_batch* batch, const void* theta_x, const void* theta_c, void* x0,
                              void* s0, void* y0, void* stream);
cosmo_status cosmo_ws_backward(cosmo_batch* batch, const void* theta_x, const void* theta_c,
                               const void* gx0, const void* gs0, const void* gy0, void* gtheta_x,
                               void* gtheta_c, void* stream);

/* Unroll K iterations from (x0, s0, y0) (NULL = zero start).
 *   sigma_host: host [K] (NULL = 1e-6 every step, the value of Sec. 2.2)
 *   rho:   dev real [K][m_total], per-row penalties before rectification
 *   alpha: dev real [K][ninst]
 *   xK, sK, yK: dev real outputs (NULL = not wanted)
 *   loss:  dev double [ninst] output ||A x^K + s^K - b||^2 + ||P x^K + q - A'y^K||^2
 *          (NULL = not wanted; required if a backward will seed from it)
 *   record_tape: 1 keeps what cosmo_backward needs (the tape), 0 does not.
 * Errors: E_INVAL (K < 1, NULL rho/alpha), E_NOMEM, E_CUDA. */
cosmo_status cosmo_forward(cosmo_batch* batch, int32_t K, const double* sigma_host,
                           const void* rho, const void* alpha, const void* x0,
                           const void* s0, const void* y0, void* xK, void* sK, void* yK,
                           double* loss, int32_t record_tape, void* stream);

/* Reverse pass of the last taped forward.  Cotangents (dev, NULL = 0):
 *   gxK, gsK, gyK: real [n_total]/[m_total]/[m_total] for x^K, s^K, y^K
 *   gloss: double [ninst] cotangent of the forward's loss
 * Outputs (dev, NULL = not wanted):
 *   grho: real [K][m_total] w.r.t. the unrectified rho
 *   galpha: real [K][ninst]
 *   gx0, gs0, gy0: real cotangents of the starting point.
 * Errors: E_STATE (no tape, or the tape was overwritten), E_INVAL, E_CUDA. */
cosmo_status cosmo_backward(cosmo_batch* batch, const void* gxK, const void* gsK,
                            const void* gyK, const double* gloss, void* grho, void* galpha,
                            void* gx0, void* gs0, void* gy0, void* stream);

/* Residuals of App. E at a point: rp2[i] = ||A x + s - b||^2,
 * rd2[i] = ||P x + q - A'y||^2, obj[i] = 1/2 x'Px + q'x (dev double [ninst],
 * each NULL = not wanted).  x, s, y: dev real. */
cosmo_status cosmo_residuals(cosmo_batch* batch, const void* x, const void* s, const void* y,
                             double* rp2, double* rd2, double* obj, void* stream);

/* Learnable per-iteration penalty (one scalar per step, shared by all rows and
 * instances) mapped to per-row values: rho[k][r] = exp(log_rho[k]) * w_r with
 * w_r = eq_scale on zero-cone rows and 1 elsewhere (the COSMO/OSQP equality
 * scaling, App. E).  log_rho: dev double [K]; rho: dev real [K][m_total]. */
cosmo_status cosmo_rho_from_log(cosmo_batch* batch, int32_t K, const double* log_rho,
                                double eq_scale, void* rho, void* stream);
/* Adjoint of cosmo_rho_from_log: glog[k] = sum_r grho[k][r] * rho[k][r]
 * (dev double [K], fixed-order reduction). */
cosmo_status cosmo_rho_from_log_backward(cosmo_batch* batch, int32_t K, const void* rho,
                                         const void* grho, double* glog, void* stream);
/* alpha[k][i] = alpha_k[k]  and its adjoint galpha_k[k] = sum_i galpha[k][i]. */
cosmo_status cosmo_alpha_broadcast(cosmo_batch* batch, int32_t K, const double* alpha_k,
                                   void* alpha, void* stream);
cosmo_status cosmo_alpha_reduce(cosmo_batch* batch, int32_t K, const void* galpha,
                                double* galpha_k, void* stream);

/* One end-to-end differentiable step on HOST buffers: copies the per-step
 * parameters (and warm start) host->device, runs cosmo_rho_from_log,
 * cosmo_alpha_broadcast, the forward with the residual loss, the backward
 * seeded with d(sum_i loss_i) = 1, the parameter adjoints, and copies the
 * loss and gradients device->host; synchronises the stream before returning.
 *   log_rho_host, alpha_k_host: host double [K]
 *   x0_host, s0_host, y0_host: host real (NULL = zero start)
 *   loss_host: host double [ninst]; glog_rho_host, galpha_k_host: host double [K]
 *   gx0_host, gs0_host, gy0_host: host real (NULL = not wanted)
 * Pinned host memory makes the copies asynchronous; pageable memory works. */
cosmo_status cosmo_step_host(cosmo_batch* batch, int32_t K, double sigma, double eq_scale,
                             const double* log_rho_host, const double* alpha_k_host,
                             const void* x0_host, const void* s0_host, const void* y0_host,
                             double* loss_host, double* glog_rho_host, double* galpha_k_host,
                             void* gx0_host, void* gs0_host, void* gy0_host, void* stream);

/* Kernel timing with CUDA events on the launching stream (not a part of the
 * method; for measurement).  kernel = NULL times every launch, "" turns
 * timing off, otherwise only launches of that kernel class are timed.
 * Classes: rho_check rho_rectify alpha_check precond rhs pcg post soc_fwd
 * psd_fwd residuals loss_seed bwd_gproj soc_bwd psd_bwd bwd_relax pcg_adj
 * bwd_solve rect_adjoint.  With CUDA graphs (options.use_graph = 1) the
 * events are recorded as event nodes of the graph and read back after each
 * replay (the next forward / backward, or cosmo_profile_read, waits for the
 * previous replay to finish); a change of what is timed drops the recorded
 * graphs, which are recorded again at the next call. */
cosmo_status cosmo_profile_enable(cosmo_batch* batch, const char* kernel);
/* Sum of the timed durations (ms) and number of timed launches of `kernel`
 * (NULL = all classes) since the last reset; synchronises on the recorded
 * events.  reset = 1 clears the accumulators. */
cosmo_status cosmo_profile_read(cosmo_batch* batch, const char* kernel, double* total_ms,
                                int64_t* launches, int32_t reset);

/* Copy per-instance flag bits (COSMO_FLAG_*) accumulated since the last
 * cosmo_status_sync into flags_host [ninst] and clear them.  Synchronises the
 * device.  Returns COSMO_OK even when flags are set. */
cosmo_status cosmo_status_sync(cosmo_batch* batch, int32_t* flags_host);

/* Device memory of the tape of a K-step forward with a tape, and of the
 * per-step parameters (states of one checkpoint segment, linear-solve
 * solutions, slacks, eigen-decompositions, checkpoints, rectified rho, the
 * preconditioner, the per-step gradient buffers): the memory cosmo_forward
 * allocates for a new K unless the caller supplies it.  Computed on the host.
 * Errors: E_INVAL. */
cosmo_status cosmo_workspace_bytes(const cosmo_batch* batch, int32_t K, size_t* bytes);

/* Caller-owned workspace for K-step forwards/backwards: ws (device memory of
 * at least cosmo_workspace_bytes(K) bytes, any alignment) holds the tape of
 * every later cosmo_forward / cosmo_policy_forward with this K, which then
 * allocates nothing (a forward with another K uses library memory again).
 * ws = NULL returns to library-owned memory.  The caller keeps ws alive and
 * untouched while the batch may use it.  Drops the current tape and recorded
 * graphs; synchronises the device.  Errors: E_INVAL (K < 1, bytes too small). */
cosmo_status cosmo_batch_set_workspace(cosmo_batch* batch, int32_t K, void* ws, size_t bytes);

/* Eigen-decomposition of every PSD block at unrolled step k of the last
 * forward that kept a tape (of the projection input of that step, Eq.
 * psd-proj), copied on `stream` into lam (device real, sum of p over blocks)
 * and U (device real, sum of p^2, column-major per block: column j is the
 * eigenvector of lam[j]); either may be NULL.  Block order as in the
 * problem.  A diagnostic of the path: an eigenvalue near zero is a kink of
 * the projection, a collapsing gap between eigenvalues the place where an
 * eigenvector-based backward fails and the Daleckii-Krein one does not.
 * With checkpointing only the steps of the segment in the buffer (the last
 * one after a forward) are available.  Errors: E_INVAL (k out of range, no
 * PSD block), E_STATE (no tape, or step k not in the buffer). */
cosmo_status cosmo_tape_eigen(cosmo_batch* batch, int32_t k, void* lam, void* U, void* stream);

/* ---- standalone kernels (each is one step of the path, usable alone) ---- */

/* Matrix-free solve of the reduced system of Sec. 2.3, Eq. (reduced):
 *     (P + sigma I + A' D(rho) A) x = rhs
 * for ninst independent blocks of a block-diagonal batch, by Jacobi-
 * preconditioned CG (App. D) with double inner products, one CTA per block.
 * Every array is caller-owned DEVICE memory; real = float (MIXED) or double
 * (FP64):
 *   col_off, row_off: int64 [ninst+1] (columns / rows of each block)
 *   A_rowptr int64 [m+1], A_col int32, A_val real: A in CSR (global indices)
 *   AT_rowptr int64 [n+1], AT_col int32, AT_val real: the CSR of A'
 *   P_rowptr int64 [n+1], P_col int32, P_val real: P (both triangles), or
 *     all three NULL for P = 0
 *   rho real [m] (> 0), rhs real [n]
 *   x real [n]: in, the warm start when warm_start = 1 (else ignored);
 *     out, the solution
 *   iters int32 [ninst] or NULL: CG iterations per block (== max_iter means
 *     the cap was reached before ||r|| <= tol ||rhs||)
 * Workspace (4n + m reals, 2 ninst int32) is allocated stream-ordered on
 * `stream` and released before return.
 * Large instances: zero-start solves of fewer than 148 instances with more
 * than 1e5 nonzeros of A each on average run a grid-wide CG instead (row and
 * column tiles spread over all SMs): through a transient cosmo_pcg_plan
 * (below) when one applies, else three kernels per iteration gathering from
 * global memory.  Both synchronise the stream before returning.  The rows of
 * instance i must only reference its own columns (other columns are dropped
 * or read as zero).  A wait that does not end within about one second
 * returns E_TIMEOUT (x is then undefined).
 * Errors: E_INVAL, E_NOMEM, E_CUDA, E_TIMEOUT. */
cosmo_status cosmo_pcg_solve(int32_t precision, int32_t ninst, int64_t n, int64_t m,
                             const int64_t* col_off, const int64_t* row_off,
                             const int64_t* A_rowptr, const int32_t* A_col, const void* A_val,
                             const int64_t* AT_rowptr, const int32_t* AT_col, const void* AT_val,
                             const int64_t* P_rowptr, const int32_t* P_col, const void* P_val,
                             double sigma, const void* rho, const void* rhs, void* x,
                             int32_t warm_start, double tol, int32_t max_iter, int32_t* iters,
                             void* stream);

/* Prepared large-instance solves of the reduced system (Sec. 2.3's
 * operator P + sigma I + A'D(rho)A at the App. B scale).  The paper has no
 * counterpart: a plan does once, per matrix, the work that does not depend
 * on rho, sigma or rhs, so that repeated solves (one per ADMM iteration, or
 * per parameter update) stream A and A' at HBM bandwidth and allocate
 * nothing.
 *
 * cosmo_pcg_plan_create copies A, A' and P (arguments as cosmo_pcg_solve,
 * device memory, values in the precision's type) into a streaming layout
 * owned by the plan: each row of A cut by column segment of its instance
 * (and each row of A' by row segment), pieces padded with zeros to a
 * multiple of 4 entries and 16-byte aligned.  The caller's arrays are not
 * used after the call returns.  Rows of instance i must reference only its
 * own columns (other entries are dropped).  Creation runs kernels on
 * `stream` and synchronises it; it needs ninst <= the device's SM count and
 * each instance's tiles to fit the kernel's shared memory, else E_INVAL
 * ("not applicable"; cosmo_pcg_solve then takes its other paths).  The plan
 * belongs to the device current at creation.  Errors: E_INVAL, E_NOMEM,
 * E_CUDA.
 *
 * cosmo_pcg_plan_solve: x = (P + sigma I + A'D(rho)A)^-1 rhs from x = 0,
 * Jacobi-PCG in its pipelined form (Ghysels & Vanroose: the iterates of
 * textbook PCG in exact arithmetic, the dot products of an iteration formed
 * alongside its matrix-vector product), stopping at ||r|| <= tol ||rhs|| or
 * max_iter iterations; rho [m], rhs [n], x [n], iters [ninst] (or NULL) as
 * in cosmo_pcg_solve.  One cooperative launch, one CTA per SM, A and A'
 * streamed by bulk asynchronous copies; the result is bitwise reproducible.
 * Synchronises the stream.  Calls on one plan must not overlap.  A wait
 * that does not end within about one second returns E_TIMEOUT (x undefined).
 * Errors: E_INVAL, E_CUDA, E_TIMEOUT. */
typedef struct cosmo_pcg_plan cosmo_pcg_plan;
typedef struct {
  int32_t nseg_a;          /* column segments of each row of A */
  int32_t nseg_at;         /* row segments of each row of A' */
  int32_t grid;            /* CTAs of the persistent launch */
  int32_t threads;         /* threads per CTA */
  int32_t cluster;         /* CTAs per thread-block cluster (one segment each) */
  int32_t ring_slots;      /* chunk buffers per streaming warp */
  int64_t layout_bytes;    /* device bytes of the streaming copies of A and A' */
  int64_t smem_bytes;      /* dynamic shared memory per CTA */
  int64_t quads_a;         /* 4-entry groups streamed per pass over A (padding included) */
  int64_t quads_at;        /* the same for A' */
} cosmo_pcg_plan_info;
cosmo_status cosmo_pcg_plan_create(int32_t precision, int32_t ninst, int64_t n, int64_t m,
                                   const int64_t* col_off, const int64_t* row_off,
                                   const int64_t* A_rowptr, const int32_t* A_col, const void* A_val,
                                   const int64_t* AT_rowptr, const int32_t* AT_col,
                                   const void* AT_val, const int64_t* P_rowptr,
                                   const int32_t* P_col, const void* P_val, cosmo_pcg_plan** out,
                                   void* stream);
cosmo_status cosmo_pcg_plan_solve(cosmo_pcg_plan* plan, double sigma, const void* rho,
                                  const void* rhs, void* x, double tol, int32_t max_iter,
                                  int32_t* iters, void* stream);
cosmo_status cosmo_pcg_plan_get_info(const cosmo_pcg_plan* plan, cosmo_pcg_plan_info* out);
cosmo_status cosmo_pcg_plan_destroy(cosmo_pcg_plan* plan);

/* Phase timer of a plan's solves (off by default; no effect on results).
 * With timing on, thread 0 of every CTA records %globaltimer at the phase
 * boundaries of the first 64 iterations, and each solve ends by reducing
 * them; cosmo_pcg_plan_get_timing then returns, per phase, the mean over
 * CTAs and iterations (mean_us) and the mean over iterations of the slowest
 * CTA (slowest_us), in microseconds, COSMO_PCG_PHASES entries each (either
 * may be NULL):
 *   0 iteration start -> the R stage (the CTA's segment of z) in shared memory
 *   1 warp 0's share of the R stream (rows of A)
 *   2 the other warps' R stream finishing, and the cluster barrier
 *   3 R epilogue (t = rho o Az of the CTA's rows, partial sums)
 *   4 R -> C grid barrier
 *   5 the C stage (t) in shared memory
 *   6 warp 0's share of the C stream (rows of A')
 *   7 the other warps' C stream finishing, and the cluster barrier
 *   8 the update of the CTA's columns
 *   9 C -> R grid barrier
 * Enabling allocates the stamp buffer (device memory of the plan).
 * Errors: E_INVAL, E_NOMEM. */
#define COSMO_PCG_PHASES 10
cosmo_status cosmo_pcg_plan_set_timing(cosmo_pcg_plan* plan, int32_t enable);
cosmo_status cosmo_pcg_plan_get_timing(const cosmo_pcg_plan* plan, double* mean_us, double* slowest_us);

/* The same solve as cosmo_pcg_solve, for callers that must not allocate device
 * memory while they run (a controller calling the solver at a fixed rate
 * cannot risk cudaMalloc's latency, implicit synchronisation or failure; a
 * host that gives the library a fixed device budget may forbid allocation).
 * The paper has no counterpart: this is an interface for such callers.
 * Arguments, layouts and results are those of cosmo_pcg_solve.  The CG
 * workspace (4n + m reals and 2 ninst int32) comes from one file-scope device
 * array of COSMO_PCG_NOALLOC_MAX_BYTES bytes, which every GPU that loads the
 * library holds until the process exits; larger problems return E_INVAL.
 * The call makes no cudaMalloc / cudaFree / allocating library call.
 * It always runs the CG as one CTA per instance over global-memory vectors
 * (cosmo_pcg_solve may pick a grid-wide CG for a few large zero-start
 * instances: the same iteration, but its reduction order, and so its
 * iteration count, can differ, and it is much faster there).
 * A solve that reached max_iter is reported only as iters[i] == max_iter:
 * the per-instance flag words live in the shared array and are not returned.
 * The first call in each CUDA context looks up the array's device address
 * with that context current and caches it per context handle, so make it
 * before any stream capture; a context created later (after cudaDeviceReset,
 * or another context the caller makes current) gets its own lookup, unless
 * the driver hands the new context the handle value of a destroyed one.
 * All calls share the array (it keeps the previous call's contents; the call
 * clears what must start at zero): calls that overlap on the GPU race on it
 * and must be ordered by the caller. */
#define COSMO_PCG_NOALLOC_MAX_BYTES (16 * 1024 * 1024)
cosmo_status cosmo_pcg_solve_noalloc(int32_t precision, int32_t ninst, int64_t n, int64_t m,
                                     const int64_t* col_off, const int64_t* row_off,
                                     const int64_t* A_rowptr, const int32_t* A_col,
                                     const void* A_val, const int64_t* AT_rowptr,
                                     const int32_t* AT_col, const void* AT_val,
                                     const int64_t* P_rowptr, const int32_t* P_col,
                                     const void* P_val, double sigma, const void* rho,
                                     const void* rhs, void* x, int32_t warm_start, double tol,
                                     int32_t max_iter, int32_t* iters, void* stream);

/* Batched PSD projection, Eq. (psd-proj), on nblk blocks given in svec form
 * (cyclic Jacobi for p <= 64, tridiagonalisation + implicit QL above).
 * Block j has order p[j] and starts at svec offset off[j] of v and out
 * (dev real, sum of p(p+1)/2 entries).  lam (dev real, sum p, may be NULL)
 * and U (dev real, sum p^2, column-major per block, may be NULL) receive the
 * eigen-decomposition.  p_host/off_host: host int32/int64 [nblk].
 * precision selects float or double.  Allocates and frees its own workspace. */
cosmo_status cosmo_psd_project(int32_t precision, int32_t nblk, const int32_t* p_host,
                               const int64_t* off_host, const void* v, void* out,
                               void* lam, void* U, void* stream);

/* Daleckii-Krein backward, Eq. (psd-cotangent-dk): out = svec(U (L o (U' smat(g) U)) U')
 * per block, with L the Loewner matrix of max(x, 0) at lam (gap threshold as
 * dk_gap_tau).  Layouts as cosmo_psd_project.  Allocates nothing. */
cosmo_status cosmo_psd_dk_backward(int32_t precision, int32_t nblk, const int32_t* p_host,
                                   const int64_t* off_host, const void* lam, const void* U,
                                   const void* g, void* out, double dk_gap_tau, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* COSMO_DU_H */
