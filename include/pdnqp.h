/*
 * pdnqp.h -- C ABI of the GB300 PDNQP solver.
 *
 * PDNQP ("PDNQP: A GPU-based Factorization-free Method for Large-scale
 * Nonconvex Quadratic Programming", Chen & Lu) finds a stationary point of
 *
 *     min  c'x + 1/2 x'Qx   s.t.  l_c <= A x <= u_c,   l_x <= x <= u_x      (Eq. qp)
 *
 * with Q symmetric and possibly indefinite, by a proximal augmented-
 * Lagrangian outer loop (Algorithm 3) whose strongly convex residual-form
 * subproblems (Eq. prox-alm-subproblem / inner-qp) are solved on the GPU by
 * restarted accelerated PDHG (Algorithm 4).  A row with l_c == u_c is an
 * equality row (A_E x = b_E); every other row is an inequality row whose
 * slack lives in [l_c, u_c] (for u_c = +inf this is A_I x >= b_I, Eq. qp).
 *
 * Conventions shared by every call:
 *   - All pointers passed to pdnqp_create / pdnqp_get / pdnqp_set_start are
 *     HOST pointers.  The library copies what it needs; the caller keeps
 *     ownership of its arrays and may free them after the call returns.
 *   - +-INFINITY marks an absent bound; any |v| >= 1e20 is treated as infinite.
 *   - CSR matrices use 0-based int32 indices, row_ptr[n_rows] == nnz, column
 *     indices in [0, n_cols).  Q must be square (n x n) and symmetric with BOTH
 *     triangles stored; duplicates are not allowed.
 *   - Return values: >= 0 is a solver status (pdnqp_solve) or success (0);
 *     < 0 is an error code.  No C++ exception crosses this boundary.  The text
 *     of the last error is available from pdnqp_last_error (per handle, or
 *     thread-local when the handle is NULL).
 *   - Every computation of the method runs in the library's CUDA kernels on
 *     the current CUDA device; there is no CPU fallback.  A missing or unusable
 *     GPU makes pdnqp_create fail with PDNQP_ERR_CUDA.
 */
#ifndef PDNQP_H
#define PDNQP_H

#include <stdint.h>

#if defined(__GNUC__)
#define PDNQP_API __attribute__((visibility("default")))
#else
#define PDNQP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Solver statuses (Algorithm 3: solved, infeasibility, limits; Algorithm 4:
 * numerical error when the rejection limit of Eq. adaptive-condition is hit). */
#define PDNQP_SOLVED 0
#define PDNQP_PRIMAL_INFEASIBLE 1
#define PDNQP_DUAL_INFEASIBLE 2
#define PDNQP_ITER_LIMIT 3
#define PDNQP_TIME_LIMIT 4
#define PDNQP_NUMERICAL_ERROR 5

/* Error codes. */
#define PDNQP_ERR_ARG (-1)           /* bad pointer, size or parameter name */
#define PDNQP_ERR_BOUNDS (-2)        /* l > u somewhere, or NaN data */
#define PDNQP_ERR_NOT_SYMMETRIC (-3) /* Q is not square/symmetric with both triangles */
#define PDNQP_ERR_CUDA (-4)          /* CUDA runtime failure (message has the detail) */
#define PDNQP_ERR_OOM (-5)           /* device allocation failed */
#define PDNQP_ERR_STATE (-6)         /* call not valid in the handle's current state */

/* Arithmetic of the hot path (option "precision"). */
#define PDNQP_FP64 64      /* plain form: every vector, matrix value and sum in FP64 */
#define PDNQP_FP32_BULK 32 /* SpMVs and vector updates in FP32; acceptance sums, restart/termination
                              reductions, multiplier/penalty updates and the proximal-shift check in FP64 */

typedef struct pdnqp pdnqp_t;

/* Host CSR matrix. */
typedef struct {
  int32_t n_rows;
  int32_t n_cols;
  int64_t nnz;
  const int32_t *row_ptr; /* n_rows + 1 entries */
  const int32_t *col_idx; /* nnz entries */
  const double *val;      /* nnz entries */
} pdnqp_csr;

/* Residuals of Eq. outer-residuals / outer-scales evaluated on the ORIGINAL
 * (unscaled) data, with variable-bound violations counted in r_p (the external
 * test of Sec. 4.1), plus counters. */
typedef struct {
  double r_p, r_d, s_p, s_d;
  double rel_kkt;            /* max(r_p / (1 + s_p), r_d / (1 + s_d)) */
  int64_t outer_iters;       /* Algorithm 3 iterations */
  int64_t inner_iters;       /* accepted Algorithm 4 iterations, all solves */
  int64_t trials;            /* trial steps (accepted + rejected) */
  int64_t restarts;
  int64_t kkt_passes;        /* inner matrix passes (3 SpMVs per trial, 2 per check) */
  double solve_seconds;      /* wall time of the last pdnqp_solve */
  double gamma;              /* proximal step of Eq. R-choice (scaled problem) */
  double lambda_min;         /* Lanczos estimate of lambda_min of the scaled Q */
  double obj;                /* c'x + 1/2 x'Qx at the returned x */
  int64_t kernel_launches;   /* CUDA kernels launched by the last pdnqp_solve (graph nodes included) */
  double inner_seconds;      /* wall time spent in the device-driven inner loops (Algorithm 4 iterations) */
  double setup_seconds;      /* wall time of the per-outer-iteration inner setup (warm start, scaling, steps) */
  double loop_seconds;       /* device time (CUDA events) of the persistent trial-loop launches; 0 in graph modes */
  int64_t loop_trials;       /* trials run inside those launches */
  int64_t loop_blocks;       /* blocks of the persistent launch (0: graph modes) */
  int64_t loop_launches;     /* persistent trial-loop launches (including ones that found nothing to do) */
  double loop_phase_seconds[6]; /* device time of their passes as seen by block 0 (globaltimer): primal work,
                                   primal barrier wait, row work, row barrier wait, column work, column barrier
                                   wait + acceptance decision */
  int64_t ctrl_used;         /* outer iterations whose rho_in / primal weight came from the learned controller */
  int64_t ctrl_fallbacks;    /* outer iterations where the paper's rule overrode it (fallback) */
} pdnqp_residuals;

/* Creation options (pdnqp_create uses precision = PDNQP_FP64, device = current,
 * stream = the legacy default stream). */
typedef struct {
  int32_t precision; /* PDNQP_FP64 or PDNQP_FP32_BULK */
  int32_t device;    /* CUDA device ordinal, or -1 for the current device */
  void *stream;      /* cudaStream_t all work is issued on; NULL = default stream */
} pdnqp_options;

/* Builds a solver for Eq. qp.  Copies and validates the inputs, orders the
 * rows equality-first, builds CSR A, A^T and Q (diagonal made explicit) on the
 * device once (Sec. 3.4, "Fixed sparse matrices"), applies the outer Ruiz
 * scaling and objective scalar (Sec. 3.1, Eq. scaled-problem) and chooses the
 * proximal step gamma (Eq. R-choice, FP64 Lanczos).  Sizes: Q is n x n, c has
 * n entries, A is m x n (m may be 0; then A may be NULL), l_c/u_c have m
 * entries, l_x/u_x n entries.  On success *out owns all device memory and 0 is
 * returned; on failure *out is NULL and a negative code is returned. */
PDNQP_API int pdnqp_create(pdnqp_t **out, const pdnqp_csr *Q, const double *c, const pdnqp_csr *A, const double *l_c,
                 const double *u_c, const double *l_x, const double *u_x);
PDNQP_API int pdnqp_create_ex(pdnqp_t **out, const pdnqp_csr *Q, const double *c, const pdnqp_csr *A, const double *l_c,
                    const double *u_c, const double *l_x, const double *u_x, const pdnqp_options *opt);

/* Frees the handle and its device memory.  NULL is accepted. */
PDNQP_API void pdnqp_destroy(pdnqp_t *h);

/* Runs Algorithm 3 (outer proximal ALM) with the GPU inner solver until the
 * unscaled residuals meet r_p <= eps_abs + eps_rel s_p and r_d <= eps_abs +
 * eps_rel s_d (Eq. outer-termination), or a limit is hit.  Starts from the
 * point given by pdnqp_set_start (default x0 = 0 projected on the box,
 * multipliers 0).  Returns a PDNQP_* status (>= 0) or an error code (< 0).
 * Calling it again restarts from the start point.  In the FP32-bulk form an
 * inner solve that reaches the rejection limit (the FP32 products no longer
 * resolve the step differences of Eq. adaptive-condition) does not end the
 * solve: its last accepted point becomes the FP64 base of the next outer
 * iteration, which re-warm-starts there with zero corrections (counted by
 * pdnqp_get_param(h, "rebases")); two in a row without an accepted iteration
 * between them, or non-finite sums, are a NUMERICAL_ERROR.  In the FP32-bulk
 * form a solve that ends in NUMERICAL_ERROR continues, with parameter
 * escalate = 1 (the
 * default), as a solve of the plain FP64 form from the same start point,
 * with the time that is left (so its result is the FP64 form's); the FP64
 * solver is built on first use from a host copy of the prepared problem that
 * FP32-bulk handles keep.  pdnqp_get then
 * reports the FP64 result, with the iteration counters and times of both
 * phases added up, and pdnqp_get_param(h, "escalated") is 1. */
PDNQP_API int pdnqp_solve(pdnqp_t *h, double eps_abs, double eps_rel);

/* The batched form: solves `count` independent problems, each with its own
 * handle (distinct handles; each created on its own stream, which
 * pdnqp_create does when no stream is given), with per-problem termination
 * (Eq. outer-termination with eps_abs / eps_rel), restarts and limits.
 * Fused form (parameter batch_fused = 1 on hs[0], the default; handles on one
 * device): the inner iterations (Algorithm 4) of all problems of one
 * precision run together in one captured CUDA graph of batch_chunk trial
 * slots, one kernel launch per phase for the whole batch (per lanes-per-row
 * group), with every problem's acceptance test, periodic check, restart and
 * inner termination taken on the device; each problem's outer iteration
 * (Algorithm 3, Sec. 3.4's CPU side) runs on a host thread of its own (one
 * per problem; `threads` is not used), which sleeps while its inner solve is
 * in the graph.  A problem keeps its solo block partition, so its results
 * are bitwise those of its solo graph-form solve.  Thread-pool form
 * (batch_fused = 0): `threads` host threads (0: min(count, 16)) run
 * pdnqp_solve on the problems, largest first, so their graph-form inner
 * solves overlap on the GPU.  In both forms every solve runs the graph form
 * (the handles' "persistent" and "autotune" parameters are set to 0 for the
 * call and restored).  status[i] receives pdnqp_solve's return for hs[i];
 * the results are read with pdnqp_get per handle.  Returns 0, or the first
 * negative code of a failed solve (the others still run to the end).  Blocks
 * until all solves have finished. */
PDNQP_API int pdnqp_solve_batch(pdnqp_t *const *hs, int count, double eps_abs, double eps_rel, int threads,
                                int *status);

/* Failure-detection self-test (no counterpart in the paper).  Makes one kind
 * of bounded device wait of the persistent trial loop run out on purpose on
 * the current device, without a fault: kind 0 = a grid barrier that one of
 * its 4 blocks never reaches (the others poll the release up to their limit),
 * kind 1 = a bulk-copy mbarrier that expects 16 bytes nothing sends.  On
 * return *gave_up is 1 when every waiter gave up with a failure and set the
 * fault flag, and *seconds (may be NULL) is the wall time of the launch
 * (about a second or a few).  The context stays usable.  Returns 0,
 * PDNQP_ERR_ARG or a CUDA error code. */
PDNQP_API int pdnqp_selftest_wait(int kind, int *gave_up, double *seconds);

/* Copies the result of the last pdnqp_solve: x (n entries, original
 * coordinates) and y (m entries, original row order, sign convention of Eq.
 * kkt-stationarity: 0 in Qx + c + A'y + N(x), so y <= 0 on rows active at
 * l_c and y >= 0 on rows active at u_c).  Any of x, y, r may be NULL. */
PDNQP_API int pdnqp_get(const pdnqp_t *h, double *x, double *y, pdnqp_residuals *r);

/* Warm start for the next pdnqp_solve (Sec. 3.2.1: user-provided x0, lambda0).
 * x0 has n entries (original coordinates) or is NULL (zero); y0 has m entries
 * in original row order and the sign convention of pdnqp_get, or is NULL. */
PDNQP_API int pdnqp_set_start(pdnqp_t *h, const double *x0, const double *y0);

/* Sets / reads an algorithm parameter (Table tab:parameters plus the
 * readings of unspecified rules).  Names: time_limit, k_out, k_in,
 * sigma_init, theta_sigma, delta_gamma, rho_in_min, rho_in_max, rho_z,
 * ruiz_outer (applies to the next pdnqp_create only; read-only here),
 * ruiz_inner, k_chk, beta_suff, beta_nec, beta_art, rej_limit, kappa_shrink,
 * delta_sigma, sigma_max, tol_floor, gamma (override, > 0; setting it
 * replaces the Lanczos choice), chunk (trial slots per CUDA-graph launch),
 * iter_budget (cap on accepted inner iterations per pdnqp_solve, summed over
 * outer iterations; ITER_LIMIT when reached), g_rows / g_cols (nonzeros per
 * lane per CSR-stream chunk in the row / column SpMV kernels: 4, 8 or 16; 0 =
 * from the mean row length), persistent (1, the default: the trials of the
 * inner loop run inside one cooperative kernel launch per check period, with
 * bounded grid barriers between the primal, row and column passes; used when
 * the device supports cooperative launches, else the graph modes below),
 * loop_blocks_per_sm (blocks per SM of that launch; 0 = as many as fit),
 * cond_graph (with persistent = 0; 1: inner loop as a device-driven CUDA
 * graph with conditional WHILE/IF nodes; 0: unrolled graph of `chunk` trial
 * slots, which profilers can inspect kernel by kernel), eps_inf (tolerance
 * of the infeasibility tests on l_inf-normalised directions; 0 = 1e-5),
 * anderson (1, the default: Anderson acceleration of the multipliers and the
 * proximal center once the primal test holds on consecutive outer
 * iterations; 0 = off), anderson_mem (stored outer iterates, 2..5),
 * controller / ctrl_explore / ctrl_seed (see pdnqp_set_controller),
 * autotune (1: when the graph form runs and g_rows / g_cols are 0, the first
 * inner solve times the row and column kernels for 4, 8 and 16 lanes per row
 * and keeps the fastest for this handle; 0, the default: the mean-row-length
 * choice), escalate (FP32-bulk handles: 1, the default, continues a solve
 * that ends in NUMERICAL_ERROR in the FP64 form, see pdnqp_solve; 0 = off),
 * batch_fused and batch_chunk (read from the first handle of a
 * pdnqp_solve_batch call: 1, the default, = the fused batched form, 0 = the
 * thread-pool form; trial slots per launch of the batched graph, default 16).
 * Read-only names for pdnqp_get_param: gamma, precision, ruiz_outer,
 * create_prepare_seconds and create_setup_seconds (wall time of
 * pdnqp_create's host preparation and device setup), lanes_rows and
 * lanes_cols (the lanes-per-row defaults in use: the setup's choice or the
 * autotuner's), escalated (1 when the last solve finished in the FP64 form),
 * batch_graph_seconds, batch_graph_launches, batch_kernel_launches and
 * batch_size (the last fused pdnqp_solve_batch over this handle's precision
 * group: device time of its graph launches, their number, the batched
 * kernels they ran and the group's problem count),
 * rebases (FP32-bulk: inner solves of the last solve that ended at the
 * rejection limit and were continued from the last accepted point as a new
 * FP64 base instead of ending the solve, see pdnqp_solve).
 * Returns PDNQP_ERR_ARG for an unknown name or an out-of-range value. */
PDNQP_API int pdnqp_set_param(pdnqp_t *h, const char *name, double value);
PDNQP_API int pdnqp_get_param(const pdnqp_t *h, const char *name, double *value);

/* Problem sizes after classification: out[0..4] = n, m, m_E, m_I, nnz(Q with
 * explicit diagonal). */
PDNQP_API int pdnqp_dims(const pdnqp_t *h, int64_t *out5);

/* Text of the last error on this handle (or of this thread when h is NULL). */
PDNQP_API const char *pdnqp_last_error(const pdnqp_t *h);

/* Test hook for per-step parity.  Performs the setup of outer iteration 0
 * from the start point and runs its inner solve (Algorithm 4) with the
 * inner termination test ignored, writing a snapshot after each of the
 * n_ckpt accepted-iteration counts in ckpt (strictly increasing, >= 1).
 * Snapshot layout, doubles: [w (dw) | y (m) | wbar (dw) | ybar (m) | omega,
 * kappa, t, t_total, trials, restarts, kkt_restart, kkt_last], with dw =
 * n + m_I + m, w = (x, s_I, r_E, r_I) and y in the outer-scaled,
 * inner-unscaled coordinates of Eq. inner-qp, rows equality-first.  snap must
 * hold n_ckpt * (2 (dw + m) + 8) doubles (host memory).  Returns the number of
 * snapshots written, or a negative code. */
PDNQP_API int pdnqp_debug_inner(pdnqp_t *h, int n_ckpt, const int64_t *ckpt, double *snap);

/* Measurement hook: replays one hot-path kernel `reps` times on the handle's
 * stream with the state left by the last solve (which & 7 = 0: the fused
 * Q/A^T SpMV + acceptance kernel, 1: the fused A SpMV + dual-step kernel, 2:
 * the primal step).  With which | 8 the launches are captured into one CUDA
 * graph, launched once and timed with CUDA events (pdnqp_replay_last_ms).
 * The replays write only trial buffers and the device state is restored.
 * Returns 0 or an error. */
PDNQP_API int pdnqp_replay_kernel(pdnqp_t *h, int which, int reps);
PDNQP_API double pdnqp_replay_last_ms(const pdnqp_t *h);

/* Algorithmic (compulsory) DRAM bytes, for the roofline: of one launch of
 * the kernel `which` (same numbering as pdnqp_replay_kernel; 3: the average
 * materialisation), of one trial of the persistent trial loop (which = 5:
 * primal, row and column passes, every array once per pass, gathers served
 * from L2), or of the graph-mode kernels of one trial together (which = -1). */
PDNQP_API int pdnqp_kernel_bytes(const pdnqp_t *h, int which, double *bytes);

/* ------------------------------------------------------------------------ */
/* External KKT test on device data.                                        */
/* ------------------------------------------------------------------------ */
/* CSR matrix whose three arrays live in DEVICE memory (same layout rules as
 * pdnqp_csr). */
typedef struct {
  int32_t n_rows;
  int32_t n_cols;
  int64_t nnz;
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const double *val;
} pdnqp_device_csr;

/* Eq. qp with every array in DEVICE memory: Q (n x n, symmetric, both
 * triangles), A (m x n) and its transpose At (n x m) -- A^T y is computed
 * row-wise from At, without atomics -- and the vectors c, l_x, u_x (n) and
 * l_c, u_c (m).  m may be 0 (A, At, l_c, u_c unused).  The caller owns all
 * arrays. */
typedef struct {
  pdnqp_device_csr Q, A, At;
  const double *c, *l_c, *u_c, *l_x, *u_x;
} pdnqp_device_problem;

/* External KKT test of Sec. 4.1 for the point (x, y) (device arrays, n and m
 * doubles, y in the sign convention of pdnqp_get): writes out[0..3] = r_p,
 * r_d, s_p, s_d of Eqs. outer-residuals / outer-scales on the given (original)
 * data, with variable-bound violations counted in r_p; out is a DEVICE
 * pointer to 4 doubles.  A point passes at tolerances (eps_a, eps_r) when
 * r_p <= eps_a + eps_r s_p and r_d <= eps_a + eps_r s_d (Eq. outer-termination).  The work is issued on `stream` (cudaStream_t,
 * NULL = legacy default stream) and the call returns after the stream has
 * finished it.  Scratch for the block partial sums (5 x 1216 doubles) is
 * allocated with cudaMalloc and freed inside the call.  Returns 0 or a
 * negative error code; the message is available from pdnqp_kkt_last_error
 * (thread-local). */
PDNQP_API int pdnqp_kkt_residuals(const pdnqp_device_problem *P, const double *x, const double *y, double *out,
                                  void *stream);
PDNQP_API const char *pdnqp_kkt_last_error(void);

/* The same external KKT test without any device allocation, for callers that
 * cannot call cudaMalloc / cudaFree: for example code running inside a
 * runtime whose memory manager owns all device memory, or latency-critical
 * loops that cannot take the device-wide synchronisation of cudaFree.  The
 * paper has no counterpart; it is a variant of pdnqp_kkt_residuals.
 * Differences from pdnqp_kkt_residuals:
 *   - Scratch: a file-scope __device__ array of 5 x 1216 doubles (48,640
 *     bytes) that every GPU loading the library holds until the process
 *     exits.  Every problem that fits the int32 CSR layout is accepted (the
 *     kernels stride over rows with at most 1216 blocks); larger ones are
 *     rejected with PDNQP_ERR_ARG and a message.
 *   - Set-up: the first call on each device looks up the device address of
 *     that array (cudaGetSymbolAddress) with the device current and keeps it
 *     for the life of the process; make that first call before any stream
 *     capture.  A cudaDeviceReset unloads the library's device code, so the
 *     kept address is no longer valid afterwards: a process that resets a
 *     device must not call this entry point on that device again.
 *   - All calls on a device share the array and it keeps the last call's
 *     contents (no clearing is needed: each call writes every entry it
 *     reads).  Calls that overlap on the GPU (other streams, other host
 *     threads) race on it and must be serialised by the caller.
 *   - Asynchronous: the work is enqueued on `stream` and the call returns
 *     without waiting; out holds the residuals once the stream has reached
 *     this work, and execution errors surface at the next synchronisation.
 * Arguments, layout and return codes are those of pdnqp_kkt_residuals. */
PDNQP_API int pdnqp_kkt_residuals_noalloc(const pdnqp_device_problem *P, const double *x, const double *y,
                                          double *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Learned controller (MLP 16 -> 64 -> 64 -> 2, GELU hidden layers).         */
/* ------------------------------------------------------------------------ */
/* The network proposes the inner tolerance factor rho_in (in place of Eq.
 * inner-tolerance-factor) and the primal weight carried into the next inner
 * solve; the paper's rules remain the fallback (pdnqp_set_controller).
 * Parameters are one flat array in this order, row-major (out x in):
 * W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2] (5,378 values,
 * pdnqp_mlp_param_count()).  Inference uses BF16 weights (uint16 bit
 * patterns) and FP32 arithmetic.  All pointers below are DEVICE pointers,
 * work is enqueued on `stream` (NULL = legacy default stream) and the calls
 * return without waiting; they return 0, PDNQP_ERR_ARG (message from
 * pdnqp_mlp_last_error) or PDNQP_ERR_CUDA (launch failure). */
PDNQP_API int pdnqp_mlp_param_count(void);
/* y[batch][2] = MLP(x[batch][16]).  cache (batch x 128 floats, or NULL)
 * receives the pre-activations of both hidden layers for pdnqp_mlp_backward. */
PDNQP_API int pdnqp_mlp_forward(const uint16_t *w_bf16, const float *x, int batch, float *y, float *cache,
                                void *stream);
/* Weighted squared error L = sum_s w_s |y_s - t_s|^2 / sum_s w_s (weight NULL:
 * all 1) into *loss (device float, or NULL) and dL/dy into dy[batch][2]. */
PDNQP_API int pdnqp_mlp_wmse(const float *y, const float *target, const float *weight, int batch, float *dy,
                             float *loss, void *stream);
/* grad[5378] = dL/dtheta for dL/dy = dy, through the BF16 weights, using the
 * cache of the forward pass.  scratch holds ceil(batch / 16) x 5378 floats
 * of per-block partial gradients (batch <= 1,048,576); the sum over blocks
 * runs in a fixed order, so the result is deterministic. */
PDNQP_API int pdnqp_mlp_backward(const uint16_t *w_bf16, const float *x, const float *cache, const float *dy,
                                 int batch, float *grad, float *scratch, void *stream);
/* One Adam step (bias-corrected, step >= 1) on the FP32 master weights w with
 * moments m, v; also rewrites w_bf16 (round to nearest even). */
PDNQP_API int pdnqp_mlp_adam(float *w, uint16_t *w_bf16, const float *grad, float *m, float *v, int step, float lr,
                             float beta1, float beta2, float eps, void *stream);
/* w_bf16[i] = round-to-nearest-even(w[i]) for i < count. */
PDNQP_API int pdnqp_mlp_to_bf16(const float *w, uint16_t *w_bf16, int count, void *stream);
PDNQP_API const char *pdnqp_mlp_last_error(void);

/* Installs the controller's weights on a handle (weights: HOST pointer to
 * pdnqp_mlp_param_count() FP32 values, copied and rounded to BF16 on the
 * device; NULL removes them).  With the parameter `controller` = 1 and
 * weights installed, every outer iteration evaluates the network on the
 * features below; its two outputs correct the rules' action a_rule (trace
 * columns 19-20): a = a_rule + out, rho_in = rho_in_min + (rho_in_max -
 * rho_in_min) * sigmoid(a[0]) and the next inner solve's starting primal
 * weight omega * exp(clamp(a[1], -1, 1)) (a network with a zero last layer
 * reproduces the rules).  The paper's rules stay the fallback and
 * overrule the network: an outer iteration after one whose proposal increased
 * the relative KKT residual uses the rules (Eq. inner-tolerance-factor, the
 * carried primal weight); so do iterations without weights or with
 * controller = 0.  The parameter ctrl_explore > 0 adds Gaussian noise of that
 * standard deviation to the actions taken (seeded by ctrl_seed), for
 * generating training trajectories.  Returns 0 or a negative error code. */
PDNQP_API int pdnqp_set_controller(pdnqp_t *h, const float *weights, int count);

/* Trace of the last pdnqp_solve, one row of PDNQP_TRACE_COLS doubles per
 * outer iteration that reached the tolerance update: [0] outer index k,
 * [1] relative KKT residual (original data) after inner solve k, [2] accepted
 * inner iterations of inner solve k, [3..18] the 16 controller features,
 * [19..20] the rules' action (logit of the rho_in fraction, log primal-weight
 * ratio = 0), [21..22] the action taken, [23] 1 if the network chose it.
 * Features: log10 of the relative primal and dual residuals (original data),
 * log10 of the scaled primal ratio r_p/s_p and of the scaled dual residual,
 * the changes of the first two since the previous outer iteration, log10 of
 * the inner absolute tolerance, log10(1 + inner iterations) and log10(1 +
 * restarts) of the inner solve, log10 of the primal weight and of gamma,
 * log10 of the proximal movement |x - z| / gamma, the rules' rho_in and the
 * ratio it is built from, log10(1 + k) and the penalty-growth flag.  Writes
 * min(n, max_rows) rows to `rows` (host) and n to *n_rows. */
#define PDNQP_TRACE_COLS 24
PDNQP_API int pdnqp_get_trace(const pdnqp_t *h, double *rows, int64_t max_rows, int64_t *n_rows);

#ifdef __cplusplus
}
#endif
#endif /* PDNQP_H */
