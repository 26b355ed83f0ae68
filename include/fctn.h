/*
 * libfctn — GB300 (sm_103a) trace-regularized FCTN completion, PAM sweep.
 *
 * C ABI.  Every entry point returns an int status (FCTN_OK = 0 on success);
 * no C++ exception crosses this boundary.  After a failure,
 * fctn_last_error() returns a message for the calling thread.
 *
 * The method (arXiv 2510.22506): an N-th order tensor X (I_1 x ... x I_N) is
 * modelled as FCTN({A_k}) with factors
 *     A_k : R_{1,k} x ... x R_{k-1,k} x I_k x R_{k,k+1} x ... x R_{k,N}
 * (FCTN format, Sec. 1; Definitions 1-3 and Property 1, Sec. 2.2), and
 *     min 1/2 ||X - FCTN(A)||_F^2 + sum_k lambda_k/2 tr(A_k(k)^T L_k A_k(k))
 *     s.t. P_Omega(X - Y) = 0                                    (Eq. 1/2)
 * is solved by proximal alternating minimisation (scheme 3): each factor is
 * the solution of the Sylvester system of Eq. 5, solved through the
 * eigenbases of L_k and of the Gram M_k M_k^T (Eqs. 7-9), then X is updated
 * in closed form (Eq. 10).  Algorithm 2 adds intermediate-tensor reuse and a
 * permuted update order (Sec. 3.3): for N >= 4 the merged tensors of one
 * half of the modes (1..N/2 or N/2+1..N) share the contraction of the other
 * half (for N = 4 the pairs of Sec. 3.3; for N >= 5 a reading of
 * Table 2), and the alternating order starts every even sweep with the
 * second half.
 *
 * Layout: all tensors are dense row-major (C order).  X and Y have shape
 * (I_1, ..., I_N).  Factor k has the shape above (A_k's own mode at position
 * k).  The observation mask is one byte per element of X (non-zero =
 * observed).  Element type is double for FCTN_FP64 and float otherwise.
 *
 * Pointers: each data-passing call takes a `where` argument:
 * FCTN_HOST (pageable or pinned host memory) or FCTN_DEVICE (device memory
 * on the handle's device).  The caller owns every buffer it passes; the
 * library copies inputs into its own device-resident state (factors, X,
 * mask, intermediate tensors, workspaces), which it owns until
 * fctn_destroy().  Results are written to caller-owned buffers.
 *
 * Concurrency: a handle is not thread-safe.  Distinct handles may be used
 * concurrently from different threads and streams.  All work of a handle is
 * ordered on the stream given at creation (NULL = the legacy default stream).
 */
#ifndef FCTN_H
#define FCTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FCTN_MAX_ORDER 8

/* status codes */
enum {
  FCTN_OK = 0,
  FCTN_E_ARG = 1,        /* invalid argument (sizes, ranks, pointers, flags)            */
  FCTN_E_OOM = 2,        /* device allocation failed                                    */
  FCTN_E_SINGULAR = 3,   /* min_ij T_ij <= 0: Eq. 5 has no unique solution this way     */
  FCTN_E_NONFINITE = 4,  /* NaN/Inf appeared in the stop-test reductions                */
  FCTN_E_TIMEOUT = 5,    /* a bounded device-side wait or iteration limit ran out       */
  FCTN_E_CUDA = 6,       /* a CUDA runtime call failed                                  */
  FCTN_E_STATE = 7,      /* call out of order (e.g. sweep before data was set)          */
  FCTN_E_UNSUPPORTED = 8 /* valid request that this library does not implement          */
};

/* arithmetic of the contractions (merged tensors, Gram, right-hand side, X update) */
enum {
  FCTN_FP64 = 0,  /* everything in double: the parity path                             */
  FCTN_FP32 = 1,  /* plain single precision on the CUDA cores                          */
  FCTN_TF32 = 2,  /* tcgen05 TF32 contractions, FP32 accumulation (the factor Grams of
                     the head-mode route stay FP32 on the CUDA cores)                */
  FCTN_BF16 = 3   /* tcgen05 BF16 contractions, FP32 accumulation.  With the head-mode
                     route (reuse, plain order, N >= 3) the right-hand-side products
                     take BF16 operands and the reconstruction F of Eq. 10 TF32;
                     otherwise split operands (v = hi + lo, three MMAs per product:
                     hi.hi + hi.lo + lo.hi)                                          */
};

/* update-order policy of Algorithm 2 ("unordered permutation" of the factors) */
enum {
  FCTN_ORDER_PLAIN = 0,     /* (1, ..., N) every sweep (Algorithm 1's order)                */
  FCTN_ORDER_ALTERNATE = 1  /* N = 4: odd sweeps (1,2,3,4), even sweeps (3,4,1,2); else plain */
};

/* sign of the periodically modified negative Laplacian L_k (Sec. 3.1) */
enum {
  FCTN_LAPLACIAN_PSD = 0,     /* diagonal 2+delta, cyclic neighbours -1 (positive definite) */
  FCTN_LAPLACIAN_PRINTED = 1  /* diagonal -2-delta, cyclic neighbours +1 (as printed)       */
};

enum { FCTN_HOST = 0, FCTN_DEVICE = 1 };

/* Formation of the Gram M_k M_k^T.  DIRECT: from the merged tensor, as in
 * Eq. 5.  FACTORED: the same matrix from the Grams of the two operands of
 * the pair form of M_k (M_k[(a, b), (jL, jR)] = sum_kappa L[a, kappa, jL]
 * R[b, kappa, jR], so G = sum_{kappa, kappa'} (L L^T) o (R R^T) blockwise);
 * it has other rounding (more cancellation) than DIRECT.  AUTO: FACTORED in
 * the FP32 / TF32 / BF16 precisions when it takes fewer multiply-adds, DIRECT
 * in FP64. */
enum { FCTN_GRAM_AUTO = 0, FCTN_GRAM_DIRECT = 1, FCTN_GRAM_FACTORED = 2 };

/* How the Sylvester equation of Eq. 5 is solved (both give its unique
 * solution, with other rounding).  EIG: Eq. 8 as printed, through the
 * eigendecomposition G = C Phi C^T (Eq. 7; Jacobi on the GPU).  CHOL: in the
 * real eigenbasis Q of L_k, Eq. 6 is block diagonal: row i of W = Q^T A
 * solves W_i (G + (lam mu_i + rho) I) = (Q^T Y)_i, one FP32 Cholesky
 * factorization per distinct mu_i (floor(I_k / 2) + 1 of them), no
 * eigendecomposition; FP32 / TF32 / BF16 and s_k <= 256 only
 * (FCTN_E_UNSUPPORTED otherwise).  A pivot that is not positive (G + c I not
 * positive definite) is FCTN_E_SINGULAR, as min T <= 0 is for EIG.  AUTO:
 * CHOL where it applies, else EIG.  The FP64 refinement (refine_steps)
 * follows either. */
enum { FCTN_SOLVE_AUTO = 0, FCTN_SOLVE_EIG = 1, FCTN_SOLVE_CHOL = 2 };

typedef struct fctn_params {
  int32_t order;                                  /* N, 2 <= N <= FCTN_MAX_ORDER       */
  int32_t precision;                              /* FCTN_FP64 / FP32 / TF32 / BF16    */
  int32_t reuse;                                  /* 1 = Algorithm 2 reuse, 0 = Alg. 1 */
  int32_t order_policy;                           /* FCTN_ORDER_*                      */
  int32_t laplacian_sign;                         /* FCTN_LAPLACIAN_*                  */
  int32_t refine_steps;                           /* Sylvester refinement steps (>= 0) */
  int64_t dims[FCTN_MAX_ORDER];                   /* I_1 .. I_N                        */
  int32_t ranks[FCTN_MAX_ORDER][FCTN_MAX_ORDER];  /* R_{a,b}; only a < b is read       */
  double lambda[FCTN_MAX_ORDER];                  /* lambda_k > 0 (Eq. 1)              */
  double delta[FCTN_MAX_ORDER];                   /* delta_k > 0 (L_k)                 */
  double rho;                                     /* proximal weight rho > 0 (Eq. 3)   */
  double extrap_alpha;  /* asymmetric extrapolation (Sec. 4.3): after each factor update */
  double extrap_beta;   /* A <- A + alpha (A - beta A^(t)); alpha = 0 turns it off       */
  int32_t gram_mode;    /* FCTN_GRAM_*: how the Gram M_k M_k^T of Eq. 5 is formed        */
  int32_t rhs_ctas;     /* launch shape of the Gram / right-hand-side kernel: about this
                           many CTAs per factor update, the columns of M_k split among
                           them; 0 = built-in rule (see fctn_autotune), <= 2432        */
  int32_t eig_max_sweeps; /* cap on the Jacobi sweeps of one Gram eigendecomposition
                             (Eq. 7); 0 = 60.  Reaching it is reported in
                             fctn_stats.eig_capped, not as an error                    */
  double eig_tol;         /* FP32 Gram eigensolver: a pair (p, q) is rotated while
                             B_pq^2 > tol^2 (|B_pp| + t)(|B_qq| + t), t the smallest
                             shift of Eq. 8.  0 = matched to refine_steps (the FP64
                             refinement of the solve removes what the eigenbasis
                             leaves): 2e-4 with two or more steps, 2e-5 with one,
                             sqrt(s) FLT_EPSILON with none                              */
  double finish_fp32_at;  /* TF32 / BF16 with the head-mode route: once a sweep's
                             rel_change <= this, or rel_change has not reached a new
                             low (1 % below the lowest) for ten sweeps (the tensor-
                             core products' rounding floor), later sweeps (fctn_complete,
                             the server) use the FP32 CUDA-core products, so that
                             rel_change can reach smaller tolerances; 0 = never         */
  int32_t tile_code;      /* launch shapes of the head-mode route (fctn_autotune_tiles),
                             0 = built-in rules.  bit 0: CUDA-core products in TF32 /
                             BF16 too; bits 1-2: pipeline stages of X_(1) M_1^T (rule,
                             2, 4, 6); bits 3-4: its K split over about (304, 152, 608,
                             76) CTAs; bits 5-6: K split of the table-driven contractions
                             over about (304, 152, 608, 1) CTAs; bit 7: programmatic
                             dependent launches in the chain of the Cholesky solve.
                             Only the summation order of the contractions changes
                             with it                                                    */
  int32_t solve_method;   /* FCTN_SOLVE_*: the solve of Eq. 5 (see above)               */
} fctn_params;

typedef struct fctn_stats {
  int64_t t;          /* completed sweeps since fctn_set_data / fctn_set_factors              */
  double rel_change;  /* ||X^{t} - X^{t-1}||_F / ||X^{t-1}||_F of the last sweep               */
  double objective;   /* Eq. 2 value after the last sweep (indicator term is 0 on D)          */
  double data_term;   /* 1/2 ||X - FCTN(A)||_F^2 after the last sweep                         */
  int32_t converged;  /* fctn_complete: 1 if rel_change <= tol was reached                    */
  int32_t status;     /* FCTN_OK or the error that stopped the run                             */
  int32_t eig_sweeps; /* Jacobi sweeps of the Gram eigensolver, max over the last sweep's k    */
  int32_t eig_capped; /* factors of the last sweep whose eigendecomposition stopped at the
                         sweep cap (eig_max_sweeps) before its stop test held; the eigenbasis
                         is then orthogonal but less exact, and the FP64 refinement of the
                         solve (refine_steps) carries the rest                                  */
} fctn_stats;

typedef struct fctn_handle fctn_handle;

/* Message of the calling thread's last failure (always NUL-terminated, may be
 * truncated to n bytes).  Returns the full message length. */
size_t fctn_last_error(char* buf, size_t n);

/* Library version string (static storage). */
const char* fctn_version(void);

/* Device bytes a handle with these parameters allocates (admission control).
 * Pure host arithmetic, no GPU needed. */
int fctn_footprint_bytes(const fctn_params* p, size_t* out_bytes);

/* Validate p, allocate the device state on the current device, build the
 * L_k eigenbases (Eq. 7, closed form of a symmetric circulant) and bind the
 * handle to `cuda_stream` (a cudaStream_t; NULL = legacy default stream). */
int fctn_create(const fctn_params* p, void* cuda_stream, fctn_handle** out);

/* Copy in the observed tensor Y and the mask Omega and set X^(1) = P_Omega(Y)
 * (Algorithms 1/2, Initialize).  Resets t, the reuse cache and the order
 * schedule.  Y: prod(dims) elements; mask: prod(dims) bytes. */
int fctn_set_data(fctn_handle* h, const void* Y, const uint8_t* mask, int where);

/* Copy in the factors A_k (array of N pointers, factor k in its FCTN shape).
 * Resets t, the reuse cache and the order schedule. */
int fctn_set_factors(fctn_handle* h, const void* const* factors, int where);

/* FCTN({A_k}) of the current factors into `out` (prod(dims) elements);
 * the contraction of the FCTN format (Sec. 1) from scratch. */
int fctn_contract(fctn_handle* h, void* out, int where);

/* Run `nsweeps` PAM sweeps (each: every factor update of Eqs. 4-9 in the
 * current order, then the X update of Eq. 10).  `stats` (may be NULL)
 * receives the state after the last sweep; this synchronises the stream. */
int fctn_pam_sweep(fctn_handle* h, int nsweeps, fctn_stats* stats);

/* Sweep until rel_change <= tol (after at least one sweep) or until the
 * handle has done max_sweeps sweeps in total; then copy X into out_X (may be
 * NULL).  tol <= 0 runs exactly up to max_sweeps. */
int fctn_complete(fctn_handle* h, double tol, int max_sweeps, void* out_X, int where, fctn_stats* stats);

/* FCTN-rank growth (Algorithms 1-2 start from all-ones ranks and grow them
 * to the maximal FCTN-rank; the schedule is the caller's).  Raises the rank
 * of every bond (a, b), a < b, to ranks[a][b] (>= the current rank; a bond
 * left unchanged keeps its factors' values).  The factors keep their entries
 * and get new slices along the grown bonds, filled with scale (2u - 1): u is
 * the (c + 1)-th output of SplitMix64 seeded with `seed`, c = k 2^40 + idx,
 * idx the row-major index of the entry in factor k's new FCTN shape, mapped
 * to [0, 1) by its top 53 bits.  X, the mask and the sweep count carry over;
 * the handle is re-planned for the new ranks (tables, buffers, graphs, warm
 * starts).  FCTN_E_ARG if a rank would shrink. */
int fctn_grow_ranks(fctn_handle* h, const int32_t ranks[FCTN_MAX_ORDER][FCTN_MAX_ORDER], double scale,
                    uint64_t seed);

/* Quality of the current X against the ground truth, as the paper evaluates
 * its results (Sec. 4): the mean over the slices spanned by modes 1 and 2
 * (the mean over i_3, ..., i_N) of PSNR with Max = 1 (slice MSE floored at
 * 1e-12) and of SSIM in its global per-slice form, with c1 = (0.01)^2,
 * c2 = (0.03)^2 and sample statistics (divisor n - 1).  `truth`: the full
 * tensor, row-major, in the compute precision (double for FCTN_FP64, float
 * otherwise), on the host or device per `where`; it is not kept.  Writes
 * *psnr and *ssim (either may be NULL) and synchronises the stream. */
int fctn_quality(fctn_handle* h, const void* truth, int where, double* psnr, double* ssim);

/* Autotuner of the launch shape (fctn_params.rhs_ctas).  For each candidate
 * value it creates a probe handle with *p and that rhs_ctas on cuda_stream,
 * copies in Y, mask and factors (as fctn_set_data / fctn_set_factors, host
 * or device per `where`), runs 2 * sweeps untimed sweeps (graph capture, and
 * eigensolver warm starts closer to a running job's) and times `sweeps`
 * sweeps with CUDA events; then destroys the probe.  *best gets the fastest
 * candidate; ms_out[i] (may be NULL) the mean sweep time of candidate i in
 * milliseconds.  cand = NULL takes the built-in candidates {96, 120, 152,
 * 192, 228, 304} (ncand is then ignored; ms_out needs 6 entries).  No existing handle changes.  Handles created with different
 * rhs_ctas give results that agree within rounding (the split changes the
 * summation order of the Gram and right-hand side).  Needs the device
 * memory of one more handle with *p (fctn_footprint_bytes); synchronises
 * cuda_stream.  Errors: FCTN_E_ARG (NULL pointers, sweeps outside [1, 1000],
 * ncand outside [1, 64], a candidate outside [0, 2432]); any error of the
 * probe's create / set / sweep calls. */
int fctn_autotune(const fctn_params* p, const void* Y, const uint8_t* mask, const void* const* factors, int where,
                  const int32_t* cand, int ncand, int sweeps, void* cuda_stream, int32_t* best, double* ms_out);

/* The autotuner of the head-mode route: times `sweeps` sweeps (after twice as
 * many untimed ones) of a probe handle per tile code in cand[0..ncand) (NULL:
 * the built-in list {0, 1, 2, 4, 8, 16, 32, 64, 96, 128, 136, 160}, one
 * choice changed per candidate, and bit 7 alone and with the two 152-CTA K
 * splits; ncand is then ignored and ms_out needs 12 entries) on the caller's
 * inputs, and returns the fastest in *best and,
 * if ms_out is not NULL, each candidate's ms per sweep.  Errors as
 * fctn_autotune; a candidate outside [0, 255] is FCTN_E_ARG. */
int fctn_autotune_tiles(const fctn_params* p, const void* Y, const uint8_t* mask, const void* const* factors,
                        int where, const int32_t* cand, int ncand, int sweeps, void* cuda_stream, int32_t* best,
                        double* ms_out);

/* Copy factor k (FCTN shape) / the completed tensor X out. */
int fctn_get_factor(fctn_handle* h, int k, void* out, int where);
int fctn_get_X(fctn_handle* h, void* out, int where);

/* Synchronise the handle's stream. */
int fctn_sync(fctn_handle* h);

/* Count of kernel launches the handle has issued so far (instrumentation). */
int fctn_launch_count(fctn_handle* h, int64_t* out);

/* Capture each distinct sweep as a CUDA graph and replay it (default: on).
 * With graphs off every kernel is launched individually. */
int fctn_set_graphs(fctn_handle* h, int enable);

/* Kernel classes for profiling. */
enum {
  FCTN_KC_MERGED = 0,   /* pair intermediates / merged tensors M_k (contractions)      */
  FCTN_KC_GRAM = 1,     /* Gram + right-hand side, split over the columns of M_k        */
  FCTN_KC_REDUCE = 2,   /* fixed-order reduction of the split partials                  */
  FCTN_KC_EIG = 3,      /* Gram eigendecomposition, or the shifted Cholesky factors     */
  FCTN_KC_SOLVE = 4,    /* Eq. 8 solve and refinement; products with the L_k basis      */
  FCTN_KC_XUPDATE = 5,  /* X update of Eq. 10 fused with F = A_k(k) M_k and the sums    */
  FCTN_KC_MISC = 6,     /* trace terms, finalisation, staging                           */
  FCTN_KC_ENV = 7,      /* Grams of the factors and their chains (Gram of M_k)          */
  FCTN_KC_RHS2 = 8,     /* right-hand sides of factors 2..N from Z (chain contractions) */
  FCTN_KC_EIGAUX = 9,   /* warm-start products and rotation application of the large
                           eigensolver (the Jacobi kernel itself is FCTN_KC_EIG)        */
  FCTN_KC_SUBST = 10,   /* Cholesky solve: triangular substitutions of each row group   */
  FCTN_KC_RESID = 11,   /* Cholesky solve: residual of Eq. 5 for the refinement         */
  FCTN_KC_COUNT = 12
};

/* Time every launch of one kernel class with CUDA events recorded on the
 * handle's stream (kernel_class = -1 turns it off).  Resets the counters.
 * While profiling is on, sweeps run without graphs. */
int fctn_profile(fctn_handle* h, int kernel_class);

/* Synchronise and report, since fctn_profile(): launches of the class, their
 * summed event time, and their algorithmic bytes and flops (what the method
 * must move / compute for those launches, not hardware counters). */
int fctn_profile_read(fctn_handle* h, int64_t* launches, double* ms, double* alg_bytes, double* alg_flops);

int fctn_destroy(fctn_handle* h);

/* ---- serving: continuous batching of completion jobs ----------------------
 * A server admits submitted jobs (any order, sizes, ranks, sampling rates)
 * while a slot is free and the job's fctn_footprint_bytes fits the memory
 * budget.  An admitted job keeps its factors, X and mask on the device; each
 * of its sweeps is one CUDA-graph launch on the job's own stream, so sweeps
 * of different jobs overlap on the GPU.  With FCTN_SERVER_GROUP the ready
 * jobs of one shape class (identical fctn_params) sweep together: their
 * sweeps are captured into one CUDA graph (each job's kernels on its own
 * stream, joined to the group's), launched again as one graph while the
 * members and their sweep signatures stay the same, and captured anew when
 * they change.  A job runs until rel_change <= tol or max_sweeps sweeps, then
 * waits (X resident) until fctn_server_result.  The caller drives the
 * scheduler with fctn_server_step (non-blocking). */
enum { FCTN_JOB_QUEUED = 0, FCTN_JOB_RUNNING = 1, FCTN_JOB_DONE = 2, FCTN_JOB_FAILED = 3 };
enum { FCTN_SERVER_GROUP = 1 };

typedef struct fctn_server_config {
  int32_t max_jobs;         /* concurrent jobs (slots), 1..1024                          */
  int32_t flags;            /* FCTN_SERVER_GROUP: grouped sweeps of same-shape jobs      */
  size_t mem_budget_bytes;  /* device bytes for admitted jobs; 0 = 80 % of free memory  */
} fctn_server_config;

typedef struct fctn_job_info {
  int32_t state;                      /* FCTN_JOB_*                                    */
  int32_t status;                     /* FCTN_OK or the error that failed the job      */
  int64_t sweeps;                     /* sweeps completed                              */
  double rel_change, objective;       /* of the last completed sweep                   */
  double t_submit, t_admit, t_done;   /* host steady-clock seconds                     */
} fctn_job_info;

typedef struct fctn_server fctn_server;

int fctn_server_create(const fctn_server_config* cfg, fctn_server** out);
/* Copy a job in (host buffers: Y, mask bytes, factors in their FCTN shape).
 * Fails with FCTN_E_OOM if the job alone exceeds the memory budget. */
int fctn_server_submit(fctn_server* s, const fctn_params* p, const void* Y, const uint8_t* mask,
                       const void* const* factors, double tol, int max_sweeps, uint64_t* job_id);
/* One scheduling pass: retire finished sweeps, launch next sweeps, admit jobs. */
int fctn_server_step(fctn_server* s, int* running, int* queued);
int fctn_server_poll(fctn_server* s, uint64_t job_id, fctn_job_info* info);
/* Copy the finished job's X out (out_X may be NULL) and release the job. */
int fctn_server_result(fctn_server* s, uint64_t job_id, void* out_X, int where);
/* Ids of jobs that finished (DONE or FAILED) since the last call, up to cap;
 * *n gets the count. */
int fctn_server_finished(fctn_server* s, uint64_t* ids, int cap, int* n);
int fctn_server_stats(fctn_server* s, int64_t* sweeps_launched, size_t* bytes_in_use);
/* Grouped sweeps so far: group-graph launches and (re)captures. */
int fctn_server_group_stats(fctn_server* s, int64_t* group_launches, int64_t* group_captures);
int fctn_server_destroy(fctn_server* s);

/* ---- FCTN contraction without device allocation --------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory: code whose GPU memory is entirely owned by
 * another allocator (for example a framework's caching allocator that has
 * reserved the device), and latency-critical loops where cudaMalloc/cudaFree
 * would synchronise the device.  It computes the same FCTN({A_k}) as
 * fctn_contract, but without a handle and without allocating: the
 * intermediates of the contraction chain live in one static device array of
 * FCTN_NOALLOC_SCRATCH_BYTES (each intermediate may use half of it), which
 * every GPU that loads this library holds until the process exits.
 *
 * order, dims[order]: N and I_1..I_N.  ranks: N*N row-major, ranks[a*N+b]
 * read for a < b.  precision: FCTN_FP64 or FCTN_FP32 (element type double /
 * float).  factors: N device pointers, factor k in its FCTN shape (mode k at
 * position k, row-major).  out: device buffer of prod(dims) elements.  All
 * work is queued on cuda_stream (NULL = legacy default stream); the call
 * returns without synchronising.
 *
 * Errors: FCTN_E_ARG for bad arguments or when an intermediate would exceed
 * half the scratch, FCTN_E_UNSUPPORTED when a chain intermediate would have
 * more indices than the planner holds (nothing is launched in either case);
 * FCTN_E_CUDA if a CUDA error from earlier work was already pending on the
 * calling thread (reported and cleared before anything is queued) or if a
 * launch fails.  Every call looks up the scratch array's device address
 * (cudaGetSymbolAddress) with the caller's device current; the first call on
 * a device may also load the library's device code, so make that first call
 * before any stream capture.  Every call on a device shares the one scratch
 * array and it keeps the last call's contents (every element a call reads is
 * written by that call first, so nothing needs clearing); calls that overlap
 * on the GPU (different streams, or host threads) race on it and must be
 * serialised by the caller. */
#define FCTN_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int fctn_contract_noalloc(int order, const int64_t* dims, const int32_t* ranks, int precision,
                          const void* const* factors, void* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FCTN_H */
