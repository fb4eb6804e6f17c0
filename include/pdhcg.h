/*
 * pdhcg.h - C ABI of the B300 restarted PDHCG solver for convex QP.
 *
 * Method: Huang, Zhang, Li, Ge, Liu, Ye, "Restarted Primal-Dual Hybrid
 * Conjugate Gradient Method for Large-Scale Quadratic Programming",
 * arXiv 2405.16160.
 *
 *   minimize 1/2 x'Qx + c'x   subject to   A x <= b          (paper Eq. (1))
 *
 * with Q symmetric positive semidefinite.  The first m_eq rows of A are
 * equalities (the "Gx = q inside Ax <= b" rows of Section 4); their
 * multipliers are free, the others are >= 0.  Every entry point returns a
 * qp_status; nothing aborts, exits or traps.  All floating point is IEEE
 * binary64.  All index arrays are int32 CSR (row pointer of length rows+1
 * starting at 0, then column indices and values in row order).
 *
 * Threading: calls on one handle must not overlap; separate handles are
 * independent.  A handle is bound to the CUDA device that was current when
 * it was created.
 */
#ifndef PDHCG_H
#define PDHCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDHCG_ABI_VERSION 2

typedef struct qp_handle qp_handle;

typedef enum {
  QP_OK = 0,
  QP_ERR_INVALID_ARG = 1,     /* a size, pointer, index or value is out of range */
  QP_ERR_OOM = 2,             /* device allocation failed */
  QP_ERR_CUDA = 3,            /* a CUDA runtime call failed (see qp_last_error) */
  QP_ERR_NOT_SOLVED = 4,      /* a result was requested before any solve */
  QP_ERR_DEVICE_TIMEOUT = 5,  /* a bounded device-side grid barrier gave up */
  QP_ERR_NO_DEVICE = 6        /* no CUDA device is visible */
} qp_status;

typedef enum {
  QP_TERM_NONE = -1,
  QP_TERM_SOLVED = 0,         /* relKKT <= tol (Section 4, progress metric) */
  QP_TERM_ITER_LIMIT = 1,
  QP_TERM_TIME_LIMIT = 2,
  QP_TERM_NUMERICAL_ERROR = 3 /* p'(Q + I/tau)p <= 0 or a non-finite value in CG */
} qp_termination;

enum { QP_CG_ADAPTIVE = 0, QP_CG_FIXED = 1 };
/* Arithmetic of the iteration.  FP64: everything in IEEE binary64.  MIXED:
 * matrix values, iterates and SpMV arithmetic in binary32; dot products
 * accumulated from exact binary32 products in double-float and combined in
 * binary64; every scalar of the method (step sizes, primal weight, CG
 * coefficients, relKKT, restart tests) in binary64.  A mixed solve ends by
 * re-evaluating its result with the binary64 data (qp_info.check_relkkt)
 * and, if refine is set and that misses tol, continuing in FP64. */
enum { QP_PREC_FP64 = 0, QP_PREC_MIXED = 1 };
enum { QP_RESTART_ADAPTIVE = 0, QP_RESTART_NONE = 2 };
/* Step size.  FIXED: eta = 1/(2||A||_2) for the whole solve (Section 3.2).
 * ADAPTIVE: the adaptive step-size rule of Section 4.  Every step is an
 * attempt from z = (x, y) with the current eta to a trial point z' (the CG
 * x-step and the dual step); with dz = z' - z, ||dz||_w^2 = omega ||dx||^2 +
 * ||dy||^2 / omega and L = ||dz||_w^2 / (2 |dy' A dx| + dx' Q dx), the attempt
 * is accepted when eta <= L, else z is kept.  Either way the next eta is
 * min((1 - (a+1)^-0.3) L, (1 + (a+1)^-0.6) eta), a = attempts so far (the
 * PDLP update the paper's rule builds on).  Averages become step-weighted
 * (sum eta_k z_k / sum eta_k); eval_freq, max_iter and qp_iterate count
 * attempts (the same as iterations with the fixed step). */
enum { QP_STEP_FIXED = 0, QP_STEP_ADAPTIVE = 1 };

/* qp_create flags */
#define QP_CREATE_CHECK_SYMMETRY 1u /* reject Q unless |Q - Q'| <= 1e-12 max|Q| entrywise */
#define QP_CREATE_SCALE 2u          /* Section 4 preprocessing: diagonal D1, D2 from 10 Ruiz
                                       steps and one Pock-Chambolle step on [[Q, A'], [A, 0]];
                                       the solver iterates on D2 Q D2, D1 A D2, D2 c, D1 b and
                                       measures relKKT on the original problem */
#define QP_CREATE_PENALTY 4u        /* Section 4 augmented penalty on the m_eq equality rows
                                       G x = q: the iteration runs on Q + rho G'G and
                                       c - rho G'q with rho = 0.1 ||Q||_2 / ||G'G||_2 (30 power
                                       iterations each; rho = 0 without equality rows); the
                                       scaling, when asked for, is computed on the penalised
                                       problem, and relKKT is always measured on the problem as
                                       given (the two share their KKT points).  qp_create
                                       returns QP_ERR_INVALID_ARG when G'G would take more than
                                       2^28 products (a dense equality row makes Q dense). */

/* debug_flags (fault injection; never used by default) */
#define QP_DEBUG_BARRIER_NEVER_RELEASES 1u /* the CG kernel's first grid barrier is never
                                              released, so its bounded wait runs out */

/*
 * Device memory and stream supplied by the caller (e.g. PyTorch's caching
 * allocator and current stream).  alloc must return 256-byte aligned device
 * memory usable on `stream`, or NULL on failure; free releases it.  A NULL
 * context, or NULL alloc/free, means cudaMalloc/cudaFree.  Every handle runs
 * its work on a non-blocking stream of its own; each call orders that stream
 * after `stream` on entry and `stream` after it on return (by events), so
 * device buffers the caller passes are read and written in the caller's
 * stream order.  A NULL stream (or a NULL context) is the legacy default
 * stream, PyTorch's default stream.
 */
typedef struct {
  void* (*alloc)(size_t bytes, void* user, void* stream);
  void (*free)(void* ptr, size_t bytes, void* user, void* stream);
  void* user;
  void* stream; /* cudaStream_t */
} qp_device_ctx;

/*
 * Solver options.  Defaults (qp_options_default) follow the paper where it
 * gives a value and the documented readings where it does not.
 */
typedef struct {
  double tol;                 /* relKKT tolerance (Section 4); default 1e-4 */
  int64_t max_iter;           /* limit on inner PDHCG iterations; default 100000 */
  double time_limit_s;        /* wall-clock limit checked between chunks; default 3600 */
  int32_t eval_freq;          /* iterations between relKKT evaluations; default 64 */
  int32_t cg_mode;            /* QP_CG_ADAPTIVE (Section 4 rule) or QP_CG_FIXED (PDHCG-fixed) */
  int32_t cg_fixed_n;         /* N for QP_CG_FIXED (Section 2); default 5 */
  int32_t cg_max;             /* cap on CG steps in adaptive mode; default 100 */
  double cg_eps_factor;       /* eps_k = eps_{k-1} + factor*relKKT (Section 4); default 0.05 */
  int32_t restart_mode;       /* QP_RESTART_ADAPTIVE or QP_RESTART_NONE */
  int32_t power_iters;        /* power iterations for ||A||_2 (Section 3.2 step); default 30 */
  double beta_suff;           /* restart parameters of Section 4: 0.2 */
  double beta_nec;            /* 0.8 */
  double beta_art;            /* 0.2 */
  double theta_pw;            /* primal weight smoothing of Section 4: 0.2 */
  double eps_zero;            /* threshold of the primal weight update; default 1e-10 */
  int32_t primal_weight_update; /* 1: update omega at restarts (Section 4); default 1 */
  int32_t warm_start;         /* 1: start from qp_set_warm_start / qp_set_state data */
  double omega0;              /* > 0 overrides omega_0 = ||c||_2/||b||_2 */
  double eta;                 /* > 0 overrides eta = 1/(2||A||_2) */
  int32_t kernel_timing;      /* 1: time every CG-kernel launch with CUDA events */
  uint32_t debug_flags;       /* QP_DEBUG_* fault injection, 0 by default */
  int32_t precision;          /* QP_PREC_FP64 (default) or QP_PREC_MIXED */
  int32_t refine;             /* mixed: continue in FP64 if the FP64 check misses tol; default 1 */
  int32_t step_mode;          /* QP_STEP_FIXED (eta = 1/(2||A||_2), Section 3.2; default) or
                                 QP_STEP_ADAPTIVE (Section 4 adaptive step size, see below) */
  int32_t mixed_stall_evals;  /* mixed with refine: once the best relKKT of the FP32 phase
                                 is below 1000 FP32 epsilons (1.2e-4), after max(this, a
                                 quarter of the evaluations so far) evaluations in a row
                                 without a 10% gain on it, the FP32 phase ends and FP64
                                 refinement continues from its iterate (an FP32 rounding
                                 floor above tol); 0: off; default 32 */
  int64_t reserved[6];
} qp_options;

/* Result of a solve (also returned by qp_get_stats). */
typedef struct {
  int32_t termination;        /* qp_termination */
  int32_t returned_avg;       /* 1: the solution is the epoch average (x~, y~) */
  int64_t iterations;         /* inner PDHCG iterations */
  int64_t cg_steps;           /* CG steps (matrix products with Q + I/tau) */
  int64_t restarts;
  int64_t evaluations;        /* relKKT evaluations (incl. the one at x0) */
  double relkkt, r_primal, r_dual, r_gap; /* of the returned iterate (Section 4) */
  double primal_obj, dual_obj;            /* 1/2x'Qx + c'x and -1/2x'Qx - b'y */
  double norm_A, eta, omega, tau, sigma;  /* final step-size state */
  double setup_ms;            /* power iteration + initial evaluation, device time */
  double solve_ms;            /* whole qp_solve wall time */
  double cg_kernel_ms;        /* kernel_timing: summed CUDA-event time of CG launches */
  int64_t cg_kernel_launches; /* kernel_timing: CG launches that did work */
  int64_t cg_kernel_spmvs;    /* kernel_timing: Q products inside those launches */
  int32_t device_error;       /* nonzero: a bounded device wait gave up */
  int32_t cooperative;        /* 1: the CG kernel ran as a cooperative launch */
  int32_t precision;          /* QP_PREC_* the solve started in */
  int32_t pad0;
  int64_t mixed_iterations;   /* mixed: iterations done in the binary32 phase */
  int64_t refine_iterations;  /* mixed: iterations of the FP64 refinement phase */
  double mixed_relkkt;        /* mixed: relKKT at the end of the binary32 phase */
  double check_relkkt;        /* mixed: relKKT of that iterate with the binary64 data */
  int64_t attempts;           /* steps tried: iterations + rejected adaptive steps */
} qp_info;

/* Scalar part of the iteration state (for checkpoint / resume and parity). */
typedef struct {
  double eta, omega;          /* tau = eta/omega, sigma = eta*omega */
  double eps;                 /* adaptive CG precision eps_k */
  double relkkt_last;         /* latest evaluated relKKT of the current iterate */
  double kkt_anchor;          /* relKKT at the epoch's restart point */
  double kkt_prev_cand;       /* candidate relKKT at the previous evaluation */
  int64_t j;                  /* iterates in the running average */
  int64_t k_total;            /* inner iterations so far */
  int64_t restarts;
  int64_t cg_total;
  int64_t attempts;           /* steps tried so far (= k_total with the fixed step) */
  double weight_sum;          /* adaptive step: sum of the accepted etas of this epoch */
} qp_state_scalars;

/* Host vectors of the iteration state; NULL entries are skipped on get and
 * read as zeros on set.  x, x_avg, x_anchor have n entries; the y's have m. */
typedef struct {
  double* x;
  double* y;
  double* x_avg;
  double* y_avg;
  double* x_anchor;
  double* y_anchor;
} qp_state_vectors;

/* One relKKT evaluation record, produced every eval_freq iterations. */
typedef struct {
  int64_t k;                  /* iteration count at the evaluation */
  double kkt_cur, kkt_avg;    /* relKKT of the current iterate and of the average */
  double omega;               /* primal weight after this evaluation */
  int32_t restart;            /* 0 none, 1 restart to current, 2 restart to average */
  int32_t cg_last;            /* CG steps of the last iteration before it */
} qp_trace_entry;

/* ---------------------------------------------------------------- lifecycle */

const char* qp_status_string(qp_status s);
int qp_abi_version(void);
/* Message of the last failed call on this thread (CUDA error text etc.). */
const char* qp_last_error(void);

void qp_options_default(qp_options* o);

/*
 * Copy a QP to the current CUDA device (paper Eq. (1)).
 * Q_*: n x n CSR, both triangles stored; A_*: m x n CSR; c: n; b: m (host
 * pointers, read only during the call; the caller keeps ownership).
 * Validation: n > 0, m >= 0, 0 <= m_eq <= m, nnz < 2^31, rowptr[0] = 0 and
 * monotone, columns in [0, cols), all values finite.  With a device visible
 * the entries are checked on it right after the copy (with QP_CREATE_PENALTY
 * or QP_CREATE_CHECK_SYMMETRY, and without a device, on the host first); the
 * error and its message are the same either way.  Duplicate (i, j) entries
 * are summed; rows are sorted.  A' is built on the device (a stable sort of
 * A's entries by column) and stored explicitly.  ctx may be NULL.
 * Errors: QP_ERR_INVALID_ARG, QP_ERR_NO_DEVICE, QP_ERR_OOM, QP_ERR_CUDA;
 * *out is NULL on failure.
 */
qp_status qp_create(qp_handle** out, int32_t n, int32_t m, int32_t m_eq,
                    const int32_t* Q_rowptr, const int32_t* Q_col, const double* Q_val,
                    const int32_t* A_rowptr, const int32_t* A_col, const double* A_val,
                    const double* c, const double* b, const qp_device_ctx* ctx,
                    uint32_t flags);

/* Free the handle and its device memory (after synchronising its stream). */
void qp_destroy(qp_handle* h);

/* ---------------------------------------------------------------- solving */

/*
 * Restarted PDHCG (Algorithm 1 with the Section 4 heuristics).  Runs on the
 * handle's stream; returns after the solve has finished.  Starts from x = y = 0
 * unless o->warm_start.  info may be NULL.  QP_OK is returned also when the
 * solve stops early: see info->termination.  QP_ERR_DEVICE_TIMEOUT when a
 * bounded device barrier gave up (the handle stays usable).
 */
qp_status qp_solve(qp_handle* h, const qp_options* o, qp_info* info);

/* Copy the iterate returned by the last qp_solve to host arrays x (n) and y
 * (m); either may be NULL.  With QP_CREATE_SCALE these are the caller's
 * variables (x = D2 x~, y = D1 y~).  QP_ERR_NOT_SOLVED before a successful
 * qp_solve and after qp_iterate or qp_set_state (read those with
 * qp_get_state). */
qp_status qp_get_solution(const qp_handle* h, double* x, double* y);

/* The diagonal scaling of QP_CREATE_SCALE: d1 (m) for constraints and d2 (n)
 * for variables (all ones without it); either may be NULL.  Host memory. */
qp_status qp_get_scaling(const qp_handle* h, double* d1, double* d2);

/* Info of the last qp_solve (QP_ERR_NOT_SOLVED before the first). */
qp_status qp_get_stats(const qp_handle* h, qp_info* info);

/* Evaluation records of the last qp_solve.  Writes up to `cap` entries and
 * stores the total count in *count. */
qp_status qp_get_trace(const qp_handle* h, qp_trace_entry* out, int64_t cap, int64_t* count);

/* ------------------------------------------------- state (checkpoint / parity) */

/* Warm start (x0, y0) in the caller's variables; NULL means zeros.  Used when
 * o->warm_start = 1:
 * the anchors become (x0, y0), the averages are empty and the step sizes
 * are recomputed by the solve's set-up. */
qp_status qp_set_warm_start(qp_handle* h, const double* x0, const double* y0);

/* Read / write the full iteration state (the solver's variables: with
 * QP_CREATE_SCALE the scaled x~, y~).  qp_set_state recomputes A x and
 * A' y on the device.  A solve with o->warm_start = 2 continues from a set
 * state without recomputing the set-up. */
qp_status qp_get_state(const qp_handle* h, const qp_state_vectors* v, qp_state_scalars* s);
qp_status qp_set_state(qp_handle* h, const qp_state_vectors* v, const qp_state_scalars* s);

/*
 * Run exactly `iters` inner PDHCG iterations (Algorithm 1 loop body: CG
 * primal step, projected dual step, averages) from the current state, with
 * no relKKT evaluation, restart or termination test.  Only o's CG settings,
 * step_mode, precision and debug_flags are used; with QP_STEP_ADAPTIVE each
 * of the `iters` is one attempt (accepted or rejected).  qp_set_state fills both precisions;
 * qp_get_state and qp_evaluate then read the precision last iterated.
 */
qp_status qp_iterate(qp_handle* h, const qp_options* o, int64_t iters);

/*
 * relKKT terms (Section 4) of the current iterate and of the running
 * average.  Each output holds {r_primal, r_dual, r_gap, relKKT, primal_obj,
 * dual_obj}; either may be NULL.  The state is not changed.
 */
qp_status qp_evaluate(qp_handle* h, double kkt_cur[6], double kkt_avg[6]);

/* Estimate ||A||_2 by `iters` power iterations on A'A from ones/sqrt(n). */
qp_status qp_norm_A(qp_handle* h, int32_t iters, double* out);

/*
 * Variable bounds lo <= x <= hi (Section 4: with box constraints the primal
 * subproblem is solved by the Barzilai-Borwein projected gradient instead of
 * CG).  lo and hi are host arrays of n entries; NULL means no bound on that
 * side, and -INFINITY / +INFINITY entries are absent bounds.  They hold for
 * every later qp_solve and qp_iterate of the handle (all absent: CG again).
 * The start point and a warm start are projected into the box and every
 * iterate stays in it.  The paper's relKKT has no bound terms; with bounds
 * r_dual measures Qx + A'y + c - lambda, where lambda are PDLP's reduced
 * costs (the gradient where both bounds are finite, its positive part with
 * only a lower bound, its negative part with only an upper one), and the
 * dual objective gains lo'lambda^+ - hi'lambda^-.  BB steps: x+ =
 * min(max(x - g/alpha, lo), hi), alpha_0 = g'Mg / g'g and then s'Ms / s's
 * (M = Q + I/tau), one product with Q per step; the adaptive rule stops when
 * the step length ||x+ - x|| is at most eps_k, the fixed rule after N steps;
 * qp_info.cg_steps counts BB steps.  With QP_CREATE_SCALE the bounds are
 * scaled with the variables.  Errors: QP_ERR_INVALID_ARG (NaN, lo > hi,
 * lo = +inf or hi = -inf).
 */
qp_status qp_set_bounds(qp_handle* h, const double* lo, const double* hi);

/* The penalty weight rho of QP_CREATE_PENALTY (Section 4, augmented penalty);
 * 0 when the flag was not given or the problem has no equality rows. */
qp_status qp_get_penalty(const qp_handle* h, double* rho);

/* ---------------------------------------------- launch-shape autotuner */

/*
 * Launch shapes of the row kernels, the CUDA products with Q, A and A' that
 * carry every step of Algorithm 1 (the CG kernel's Q p, the dual step's
 * A x+, the A'y+ kernel, the relKKT products).  Index [p][k]: p = 0 FP64,
 * 1 FP32 (mixed precision); k = 0 Q, 1 A, 2 A'.
 *   lanes        lanes per row in use: G threads share one CSR row, so a
 *                warp takes 32 / G rows at a time; rows longer than 16 G
 *                entries (64 at least in FP64) go to one whole warp each
 *   lanes_rule   the choice of qp_create's rule: by the mean row length (over
 *                the rows of at most 64 entries when some are longer); FP32 Q,
 *                whose products run in the CG kernel, takes the fewest lanes G
 *                with a mean of at most 8 G entries
 *   layout       how rows go to warps: 0 groups of 32 / G rows across the grid
 *                in turn (the default for A and A'), 1 a contiguous range per
 *                warp (the default for Q), 2 a contiguous range per block whose
 *                groups its warps take in turn
 *   product_us   one product at the shape in use, microseconds (qp_tune's
 *                best-of-three timing; 0 before qp_tune)
 *   product_us_rule  the same product at the rule's lanes and layout
 *   waves        grid of the non-persistent row kernels in waves of
 *                co-resident blocks (1 at qp_create)
 *   waves_us[w]  qp_tune: the three products of the mixed path (Q, A, A'
 *                at the chosen lanes) with 1, 2 and 4 waves, microseconds
 *   tuned        1 once qp_tune has run
 */
typedef struct {
  int32_t lanes[2][3];
  int32_t lanes_rule[2][3];
  int32_t layout[2][3];
  double product_us[2][3];
  double product_us_rule[2][3];
  int32_t waves;
  int32_t tuned;
  double waves_us[3];
} qp_shapes;

/*
 * Autotuner.  Times, on this handle's own matrices, one product with each of
 * Q, A and A' in both precisions at 1, 2, 4, 8 and 32 lanes per row (each
 * with its own medium-row table) and, for A and A', each row layout (Q keeps
 * the warp ranges, the layout of its persistent CG kernel), then the row
 * kernels' grid at 1, 2 and 4 waves, and keeps the fastest shape of each (the
 * rule's unless another is faster by more than 1%).  Each timing is the best of three runs of `reps` products (reps in
 * 1..1000) on scratch vectors the call allocates and frees; the iterate,
 * warm start, bounds and statistics of the handle are left as they were.
 * The solve graphs captured so far are rebuilt by the next qp_solve.  The
 * shapes in use afterwards are written to *out (may be NULL) and returned
 * by qp_get_shapes.  Errors: QP_ERR_INVALID_ARG, QP_ERR_OOM, QP_ERR_CUDA.
 */
qp_status qp_tune(qp_handle* h, int32_t reps, qp_shapes* out);

/* The launch shapes in use (qp_create's rule, or qp_tune's choice). */
qp_status qp_get_shapes(const qp_handle* h, qp_shapes* out);

/* ------------------------------------------------------- diagnostics */

/*
 * The random-gather ceiling of the current device, measured: the best of
 * `reps` timed launches of a kernel that only sums v[idx[k]] over `count`
 * pseudo-random indices (a mix of seed and k) into an L2-resident vector of
 * n floats, with four reads in flight per thread, written to *gathers_per_s.
 * Uniformly random columns make every SpMV of the method read one 32-byte
 * sector per stored entry, so this rate, not DRAM bandwidth, bounds them;
 * benchmarks report the kernels against it.  Not part of a solve: it
 * allocates its own device buffers (cudaMalloc) and frees them.  Errors:
 * QP_ERR_INVALID_ARG, QP_ERR_NO_DEVICE, QP_ERR_OOM, QP_ERR_CUDA.
 */
qp_status qp_gather_rate(int64_t count, int32_t n, int32_t reps, uint64_t seed,
                         double* gathers_per_s);

/* ------------------------------------------------- allocation-free variant */

/* Capacity, in doubles, of the static device scratch of qp_norm_A_static (8 MiB). */
#define QP_NORM_A_STATIC_MAX_DOUBLES (1u << 20)

/*
 * The paper has no counterpart of this entry point; it serves callers that
 * cannot allocate device memory at all - a control loop held to a device
 * memory budget fixed at start-up, code running while another framework
 * owns every byte of device memory, or code that must not risk the
 * device-wide synchronisation an allocation can cause.
 *
 * Computes the same estimate as qp_norm_A: `iters` power iterations on A'A
 * from ones/sqrt(n), writing ||A||_2 to norm_out (device pointer, one
 * double) in stream order on `stream` (cudaStream_t; NULL = legacy default
 * stream).  It calls no cudaMalloc, cudaFree or other allocating routine:
 * its work vectors live in one static __device__ array of
 * QP_NORM_A_STATIC_MAX_DOUBLES doubles that every GPU loading this library
 * holds until the process exits.
 *
 * Inputs are device arrays the caller owns: A (m x n CSR, nnz entries) and
 * its transpose At (n x m CSR), both valid as qp_csr_validate would check
 * (not re-checked here); nnz only selects lanes per row.  Sizes with
 * 2n + m > QP_NORM_A_STATIC_MAX_DOUBLES - 1185 are rejected with
 * QP_ERR_INVALID_ARG and a message in qp_last_error.
 *
 * The first call on each device resolves the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the one array and it keeps
 * the last call's contents; every value a call reads is written earlier by
 * the same call.  Calls whose work overlaps on the GPU (other streams,
 * other threads) race on the array: serialise them.
 */
qp_status qp_norm_A_static(int32_t m, int32_t n, int64_t nnz, const int32_t* A_rowptr,
                           const int32_t* A_col, const double* A_val, const int32_t* At_rowptr,
                           const int32_t* At_col, const double* At_val, int32_t iters,
                           double* norm_out, void* stream);

/* ------------------------------------------------- host-only helpers (no GPU) */

/*
 * Validate a CSR matrix (rows x cols): rowptr[0] = 0, monotone, nnz =
 * rowptr[rows] < 2^31, columns in range, values finite.  Host pointers.
 */
qp_status qp_csr_validate(int32_t rows, int32_t cols, const int32_t* rowptr,
                          const int32_t* col, const double* val);

/*
 * Transpose a valid CSR matrix (rows x cols) into caller-allocated arrays
 * t_rowptr[cols + 1], t_col[nnz], t_val[nnz] with a stable counting sort:
 * within each output row the entries keep the input row order.
 */
qp_status qp_csr_transpose(int32_t rows, int32_t cols, const int32_t* rowptr,
                           const int32_t* col, const double* val, int32_t* t_rowptr,
                           int32_t* t_col, double* t_val);

/* ------------------------------------------------- batched small QPs */
/*
 * Many independent QPs solved in one persistent launch, one thread block per
 * instance, each with its own restart, primal-weight and CG-precision state
 * (Algorithm 1 with the Section 4 heuristics, the same readings as
 * qp_solve).  Each instance has Q = F F' + diag(qd), the low-rank-plus-
 * diagonal form whose products cost 2nk (the P'P acceleration of Section
 * 5.2).  An instance's vectors live in shared memory when the largest
 * instance of its size bin fits one block (about 225 KB on B300), else in a
 * per-block slice of global memory: in FP64 (9 n + 6 m + k doubles, 11 n +
 * 8 m + k with the adaptive step size), or in mixed precision FP64 iterates,
 * averages and restart points with FP32 attempt vectors (7 n + 5.5 m + 1.5 k
 * doubles).  No diagonal scaling.
 */
typedef struct qp_batch qp_batch;

/* One instance (host pointers, read during qp_batch_create only).
 * F: n x k row-major (NULL when k = 0); qd: n; A: m x n CSR with the first
 * m_eq rows equalities (validated and canonicalised like qp_create's); c: n;
 * b: m. */
typedef struct {
  int32_t n, m, m_eq, k;
  const double* F;
  const double* qd;
  const int32_t* A_rowptr;
  const int32_t* A_col;
  const double* A_val;
  const double* c;
  const double* b;
} qp_instance;

/* Per-instance outcome of the last qp_batch_solve. */
typedef struct {
  int32_t termination;        /* QP_TERM_* */
  int32_t returned_avg;       /* 1 if the returned iterate is the average */
  int64_t iterations, cg_steps, restarts;
  double r_primal, r_dual, r_gap, relkkt, primal_obj, dual_obj;  /* FP64 data */
  double eta, omega, norm_A;
  int64_t attempts;           /* steps tried (adaptive step: iterations + rejections) */
} qp_instance_result;

/* Copy count instances to the current device.  Errors: QP_ERR_INVALID_ARG
 * (bad sizes or CSR, non-finite values, an instance too large for one
 * block), QP_ERR_NO_DEVICE, QP_ERR_OOM, QP_ERR_CUDA; *out is NULL on failure. */
qp_status qp_batch_create(qp_batch** out, int32_t count, const qp_instance* inst,
                          const qp_device_ctx* ctx, uint32_t flags);
void qp_batch_destroy(qp_batch* bt);

/* Solve every instance with the same options (tol, max_iter, eval_freq, the
 * CG, restart and primal-weight settings, power_iters, omega0, eta,
 * precision; warm_start = 1 starts from qp_batch_set_warm_start's data).
 * One kernel launch; *device_ms (may be NULL) receives its CUDA-event time.
 * Per-instance outcomes: qp_batch_results. */
qp_status qp_batch_solve(qp_batch* bt, const qp_options* o, double* device_ms);

/* count entries. */
qp_status qp_batch_results(const qp_batch* bt, qp_instance_result* out);

/* The returned iterates, packed in instance order: x has sum n_i entries, y
 * sum m_i; either may be NULL. */
qp_status qp_batch_solution(const qp_batch* bt, double* x, double* y);

/* Packed start points for warm_start = 1 (NULL: zeros). */
qp_status qp_batch_set_warm_start(qp_batch* bt, const double* x0, const double* y0);

/*
 * Packed variable bounds lo <= x <= hi for every instance (host arrays of
 * sum n_i entries in instance order; NULL means no bound on that side,
 * -INFINITY / +INFINITY entries are absent bounds), as qp_set_bounds for one
 * problem (Section 4): every x-step of an instance with a finite bound is the
 * Barzilai-Borwein projected gradient, its start points are projected into
 * the box, and its relKKT uses the reduced costs; instances whose bounds are
 * all absent keep CG.  They hold for
 * every later qp_batch_solve (all absent: CG again).  Errors:
 * QP_ERR_INVALID_ARG (NaN, lo > hi, lo = +inf or hi = -inf), QP_ERR_OOM,
 * QP_ERR_CUDA.
 */
qp_status qp_batch_set_bounds(qp_batch* bt, const double* lo, const double* hi);

/*
 * The same bounds from one host array per instance instead of packed ones:
 * lo and hi are NULL (no bound on that side for any instance) or arrays of
 * count pointers, entry i NULL (instance i has no bound on that side) or n_i
 * values.  The arrays are read during the call only and copied to the device
 * through pinned staging without a packed host copy.  Errors as
 * qp_batch_set_bounds (the bad variable reported by its packed index).
 */
qp_status qp_batch_set_bounds_each(qp_batch* bt, const double* const* lo,
                                   const double* const* hi);

/* qp_batch_create groups the instances by size (n, largest first) into up
 * to 4 bins of equal count; each bin is one launch on its own stream, with
 * shared memory and block size fitted to its largest instance.
 * qp_batch_set_threads sets every bin's threads per block: 0 restores the
 * built-in default (the smallest of 64, 128, 256, 512 that keeps about 16
 * warps per SM resident given the bin's shared memory per block, and at
 * least n/8 threads: 64 up to n ~ 130, 128 up to n ~ 900, 512 at n = 2000
 * with m ~ 30); otherwise 64, 128, 256 or 512.  Results can differ from another block size in the last bits (the
 * reduction trees differ); a fixed configuration is bit-reproducible. */
qp_status qp_batch_set_threads(qp_batch* bt, int32_t threads);

/* Autotuner: the bins run concurrently and share the SMs, so every
 * candidate is timed on the whole batch: a bounded solve (o with max_iter
 * capped at sample_iters) of each bin's first sample_count instances.  Bin
 * by bin (largest instances first), each block size is tried with the other
 * bins at their current choice and the fastest is kept.  *threads_out (may
 * be NULL) receives the choice for the bin of the largest instances.  The
 * sample must fill the GPU (a few blocks per SM, and several waves) for the
 * timing to reflect throughput; sample_count >= the bin sizes takes every
 * instance. */
qp_status qp_batch_tune(qp_batch* bt, const qp_options* o, int32_t sample_count,
                        int32_t sample_iters, int32_t* threads_out);

/* ------------------------------------------------ learned warm start (MLP) */
/*
 * The network of the learned warm start (not in the paper): a multilayer
 * perceptron mapping an instance's parameters to a starting point (x0, y0)
 * for qp_batch_set_warm_start / qp_set_warm_start.  widths[0] inputs,
 * widths[n_layers] outputs, ReLU after every layer but the last; layer l is
 * z = a W_l + b_l with W_l row-major (widths[l-1] x widths[l]).  FP32
 * parameters packed in layer order, each layer W then b.  Activations are
 * row-major, one sample per row.  The loss is the weighted squared error
 * (1/B) sum_r sum_j w_j (out_rj - target_rj)^2, trained with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  in, out, target, w and grad are
 * device pointers; params of set/get are host pointers.
 */
typedef struct qp_mlp qp_mlp;

/* n_layers in [1, 16], widths in [1, 2^20]; batches of up to max_batch rows.
 * Parameters start at zero (set them with qp_mlp_set_params). */
qp_status qp_mlp_create(qp_mlp** out, int32_t n_layers, const int32_t* widths,
                        int32_t max_batch, const qp_device_ctx* ctx);
void qp_mlp_destroy(qp_mlp* net);
int64_t qp_mlp_param_count(const qp_mlp* net);
/* Host copy in/out of the packed parameters; set also resets Adam's state. */
qp_status qp_mlp_set_params(qp_mlp* net, const float* params);
qp_status qp_mlp_get_params(const qp_mlp* net, float* params);
/* out (batch x widths[n_layers]) = net(in (batch x widths[0])). */
qp_status qp_mlp_forward(qp_mlp* net, int32_t batch, const float* in, float* out);
/* The loss on one batch and its gradient (kept for qp_mlp_adam_step; also
 * copied to grad, param_count floats, when grad is not NULL).  w: per-output
 * weights or NULL for ones.  *loss (host, may be NULL) waits for the result. */
qp_status qp_mlp_loss_grad(qp_mlp* net, int32_t batch, const float* in, const float* target,
                           const float* w, float* grad, double* loss);
/* One Adam step with the gradient of the last qp_mlp_loss_grad. */
qp_status qp_mlp_adam_step(qp_mlp* net, float lr);

#ifdef __cplusplus
}
#endif

#endif /* PDHCG_H */
