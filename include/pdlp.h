/*
 * pdlp.h -- C ABI of the GB300 (sm_103a) PDLP library.
 *
 * The library solves the LP relaxation of a MIP,
 *
 *     min c^T x   s.t.  row i of A x  (<=, >=, =)  b_i,   l <= x <= u,          (eq. 1)
 *
 * (Kempke & Koch, "Fix-and-Propagate Heuristics Using Low-Precision First-Order
 * LP Solutions for Large-Scale MILP", section 1, eq. 1; the paper states the
 * rows as A x <= b, the sense per row generalises that) with restarted,
 * diagonally preconditioned PDHG ("PDLP", abstract and section 2) to a
 * RELATIVE tolerance (section 4, "Hardware and software": relative primal,
 * dual and gap tolerances; 1e-4 and 1e-6 are the paper's settings).  The
 * solution then ranks and drives the fixings of the fix-and-propagate
 * heuristic (section 2), exposed here as fp_run().
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are CSR: row_ptr[m+1] (int64, row_ptr[0] = 0, non-decreasing),
 *    col[nnz] (int32, 0 <= col < n, no duplicate (row, col) pair), val[nnz]
 *    (float64).  Column order inside a row is free.
 *  - sense[m] holds the bytes 'L' (<=), 'G' (>=) or 'E' (=).
 *  - Infinite bounds are +-INFINITY; l_j <= u_j is required.
 *  - Dual sign convention of every output: y_i <= 0 on 'L' rows, y_i >= 0 on
 *    'G' rows, free on 'E' rows; reduced costs are lambda = c - A^T y.  These
 *    are the signs the Dual and RedCost fixing strategies (section 2) read.
 *  - Ownership: the library owns nothing it returns.  Every output goes into a
 *    caller-allocated buffer; inputs are only read (host inputs are copied to
 *    the device, device inputs are read in place).
 *  - Return codes: 0 (PDLP_OK) or a negative PDLP_ERR_* value.  The solver
 *    outcome (tolerance met, iteration limit, ...) is pdlp_result.status,
 *    never the return code.  pdlp_error_string() names every code.
 *  - Reentrancy: calls share no mutable state but two mutex-guarded caches
 *    (the executable CUDA graphs of recent check periods, keyed by every
 *    launch parameter including the workspace addresses, and the autotuner's
 *    lanes per shape) and the static scratch array of
 *    pdlp_solve_device_noalloc (its note below); concurrent calls on different
 *    streams into different workspaces are independent.
 *
 * Relative KKT measures reported in pdlp_result (the definition every result
 * is judged by), for x in [l,u] and y in the dual cone, on the original data:
 *    r_p = violation of each row (only the violated side of inequalities),
 *    r_d_j = lambda_j^+ if l_j = -inf  plus  lambda_j^- if u_j = +inf,
 *    dual objective = b^T y + sum_{l_j finite} l_j lambda_j^+ - sum_{u_j finite} u_j lambda_j^-,
 *    rel_primal_res = ||r_p||_2 / (1 + ||b||_2),  rel_dual_res = ||r_d||_2 / (1 + ||c||_2),
 *    rel_gap = |c^T x - dual| / (1 + |c^T x| + |dual|),
 *    rel_kkt = max of the three.  Status PDLP_OPTIMAL means rel_kkt <= tol.
 */
#ifndef PDLP_H
#define PDLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define PDLP_OK 0
#define PDLP_ERR_INVALID_INPUT (-1) /* bad CSR, NaN, l > u, unknown sense, bad params */
#define PDLP_ERR_CUDA (-2)          /* a CUDA runtime call failed (message: pdlp_last_error) */
#define PDLP_ERR_OOM (-3)           /* device allocation failed or workspace too small */
#define PDLP_ERR_TIMEOUT (-4)       /* a bounded device-side wait gave up */
#define PDLP_ERR_UNSUPPORTED (-5)   /* requested mode not available for this input */

/* ---- solver outcome (pdlp_result.status) ----------------------------- */
#define PDLP_OPTIMAL 1      /* rel_kkt <= tol */
#define PDLP_ITER_LIMIT 2   /* iter_limit accepted iterations reached */
#define PDLP_TIME_LIMIT 3   /* time_limit_s reached */
#define PDLP_NUMERICAL 4    /* a NaN / Inf appeared in the iteration */
/* Certificates (pdlp_params.detect_infeasibility).  The paper's heuristic stops
 * when an LP has no solution (section 2); the test is PDLP's, on the movement of
 * the iterate since the last restart, at each KKT check after the tolerance test:
 * y^ = that movement of y projected onto the dual cone, lambda^ = -A^T y^ (in the
 * >=-form), d^ = b^T y^ plus the finite-bound terms of lambda^; x^ = that movement
 * of x projected onto the recession cone of [l, u]. */
#define PDLP_PRIMAL_INFEASIBLE 5 /* d^ > 0 (beyond the rounding of its terms: d^ >
                                    1e-9 x the sum of their magnitudes) and the part of
                                    lambda^ against infinite bounds has 2-norm <= 1e-8 d^:
                                    no x satisfies the rows within [l, u].  y_out holds
                                    y^ in the caller's sign convention (Farkas ray) */
#define PDLP_DUAL_INFEASIBLE 6   /* c^T x^ < 0 beyond rounding and the rows' violation by
                                    x^ (max(0, -(Kx^)_i) on inequalities, |(Kx^)_i| on
                                    equalities) has 2-norm <= 1e-8 |c^T x^|: the LP is
                                    unbounded if it is feasible.  x_out holds x^ */

/* ---- precision modes (pdlp_params.precision) -------------------------
 * PDLP_FP64:      iterates, SpMV and reductions in float64 on the explicitly
 *                 scaled matrix D_r K D_c (the parity mode).
 * PDLP_FP32:      iterates, SpMV and accumulation in float32 on the scaled
 *                 matrix stored in float32; KKT checks, restarts and the
 *                 primal weight in float64 on the float64 data.
 * PDLP_FP32_BF16A:float32 iterates on the UNSCALED matrix stored in bfloat16
 *                 (or as a bare sparsity pattern when every value is 1),
 *                 with the scaling folded into per-element step sizes
 *                 tau_j = (eta/omega) D_c,j^2, sigma_i = eta omega D_r,i^2.
 *                 Chosen only when every value is exactly representable in
 *                 bfloat16; otherwise the solver falls back to PDLP_FP32 and
 *                 reports it in pdlp_result.precision_used. */
#define PDLP_FP64 0
#define PDLP_FP32 1
#define PDLP_FP32_BF16A 2
/* values reported in pdlp_result.precision_used (PDLP_FP64/FP32 as above) */
#define PDLP_USED_BF16 2
#define PDLP_USED_PATTERN 3

typedef struct {
  int32_t m, n;
  int64_t nnz;
  const int64_t* row_ptr; /* [m+1] */
  const int32_t* col;     /* [nnz] */
  const double* val;      /* [nnz] */
} pdlp_csr;

typedef struct {
  size_t struct_size;   /* sizeof(pdlp_params); set by pdlp_default_params */
  double tol;           /* relative KKT tolerance, default 1e-4 */
  int64_t iter_limit;   /* accepted PDHG iterations, default 1000000 */
  double time_limit_s;  /* wall-clock limit of the iteration phase, default 3600 */
  int precision;        /* PDLP_FP64 (default) | PDLP_FP32 | PDLP_FP32_BF16A */
  int check_period;     /* accepted iterations between KKT checks, default 64 */
  int ruiz_iters;       /* Ruiz equilibration passes, default 10 */
  double pc_alpha;      /* Pock-Chambolle exponent, default 1; < 0 disables the pass */
  int adaptive_step;    /* 1 (default): adaptive step-size rule; 0: fixed eta, every step accepted */
  int restarts;         /* 1 (default): KKT-based restarts and primal-weight updates */
  double fixed_eta;     /* > 0 overrides the initial step size eta0 */
  double fixed_omega;   /* > 0 overrides the initial primal weight omega0 */
  int terminate;        /* 1 (default): stop at tol; 0: run to iter_limit */
  int lanes_A;          /* SpMV lanes per row of A in the step kernels (0 = automatic:
                           float32 iterates with persistent = 0 take 1 when an average
                           row has at most 8 entries; 1, 2, 4, 8, 16, 32; 1 -- each
                           thread sums and finishes whole rows -- only with
                           persistent = 0) */
  int lanes_AT;         /* SpMV lanes per row of A^T in the step kernels (as lanes_A) */
  int lanes_kkt_A;      /* lanes per row of A in the float64 KKT pass (0 = automatic;
                           2, 4, 8, 16, 32) */
  int lanes_kkt_AT;     /* lanes per row of A^T in the float64 KKT pass (as lanes_kkt_A) */
  int verbose;          /* 0 quiet; 1 one line per KKT check on stderr; 2 also the host-side
                           time of each setup phase (synchronising the stream at each) */
  int persistent;       /* 1: the step attempts of a check period run in one cooperative
                           kernel with grid-wide barriers; 2: one block per check period
                           (small LPs, such as the 200 x 400 relaxations: no launch per
                           attempt), which copies the LP into shared memory when it fits
                           and otherwise runs the cooperative kernel as one block; 0
                           (default): two kernel launches per attempt.  Same iteration
                           either way.  Batches: 1 runs one cooperative kernel per check
                           period over every LP of the batch (three grid barriers per
                           attempt); 2 is rejected. */
  int autotune;         /* 1: before iterating, time whole step attempts (primal kernel,
                           dual kernel and decision) with 1 (float32 iterates and
                           persistent = 0 only), 2, 4, 8, 16 and 32 lanes per row,
                           first for the primal kernel's A^T, then for the dual kernel's A,
                           on this LP without moving the iterate, and keep the fastest;
                           cached per (device, precision mode, m, n, nnz) for the process.
                           Lanes set explicitly in lanes_A / lanes_AT are kept.  0
                           (default): size heuristic. */
  int detect_infeasibility; /* 1 (default): test the two certificates above at each KKT
                           check (with terminate = 1); 0: never (an infeasible LP runs to
                           its iteration or time limit) */
  int debug_skip_barrier; /* fault-handling tests only (default 0): with persistent = 1,
                           block 0 of the persistent step kernel skips its grid-barrier
                           arrivals, so every block's bounded wait (2^16 polls in this
                           mode, 2^23 otherwise) runs out; the kernel records the failure
                           and returns, and the call returns PDLP_ERR_TIMEOUT with the
                           device context intact */
  int tiles;            /* float32 iterates (PDLP_FP32, PDLP_FP32_BF16A): 1 runs the
                           step attempts with the staged tile kernels -- each block streams
                           work items of at most 256 rows and 1280 nonzeros (rows longer
                           than 256 entries in slices) into shared memory with bulk copies,
                           gathers from the staged indices and sums each row in storage
                           order; 2 runs the warp-tile kernels -- every warp owns work
                           items of at most 32 rows and 64-256 nonzeros (longer rows in
                           slices) and works through them without block-wide
                           synchronisation; 0 (default) uses the lanes-per-row kernels
                           (lanes_A, lanes_AT).
                           Same iteration either way; float32 sums differ in rounding.
                           Ignored in float64 and with persistent != 0. */
  int bound_objective_rescaling; /* 1: after the Ruiz / Pock-Chambolle scaling divide the
                           objective by gamma = 1 + ||c~||_2 and the right-hand side and
                           the variable bounds by beta = 1 + ||q~||_2 (one of PDLP's
                           algorithmic variants; the paper is silent).  Without restarts
                           it is the same iteration (x~ = beta x', y~ = gamma y',
                           omega' = omega beta / gamma); the restart metric then weighs its
                           gap term by 1 / (beta gamma).  0 (default): off.  Single LPs
                           only: a batch with 1 is rejected. */
  int halpern;          /* 1: reflected restarted Halpern PDHG (one of PDLP's algorithmic
                           variants; the paper is silent): a constant step
                           eta = 0.998 / L, L the power-iteration estimate of ||K~||_2
                           (64 passes of v <- K~^T K~ v / ||K~^T K~ v|| from
                           v = 1/sqrt(n); fixed_eta > 0 overrides); each step maps the
                           Halpern iterate z through the PDHG operator T and takes
                           z' = (k+1)/(k+2) ((1+rho) T(z) - rho z) + 1/(k+2) z_a, z_a the
                           anchor (the start, then the last restart point), k the steps
                           since the last restart; no averages; the checks evaluate and
                           the solver returns the latest T(z); restarts apply the KKT
                           restart thresholds (0.2, 0.8, 0.36) to the fixed-point residual
                           ||z - T(z)||_P against the epoch's first, and move the anchor
                           and the iterate to T(z).  The decision trace records the
                           residual in place of eta_bar.  0 (default): off.  Single LPs
                           with persistent = 0 and tiles = 0 only; adaptive_step is
                           ignored. */
  double halpern_reflection; /* rho of the Halpern variant, in [0, 1]: 1 (default)
                           reflected, 0 plain Halpern */
  int restart_metric;   /* 0 (default): KKT restarts on the scaled KKT_omega; 1: the
                           normalized duality gap of the original PDLP (one of its
                           algorithmic variants; the paper is silent): for the current and
                           the average point z, r = ||z - z_last||_omega (omega-weighted,
                           scaled), rho = the maximum of the Lagrangian gap
                           L(x, y^) - L(x^, y) over the points of X x Y within r of z,
                           divided by r (by bisection on the step of the projected
                           gradient path: 6 steps on its exponent, 44 halvings); the
                           candidate with the smaller rho, the same three thresholds,
                           and the restart point's rho as the next reference.  Adds 53
                           small launches per KKT check.  Single LPs without halpern and
                           bound_objective_rescaling only. */
} pdlp_params;

typedef struct {
  int status;             /* PDLP_OPTIMAL, PDLP_ITER_LIMIT, PDLP_TIME_LIMIT, PDLP_NUMERICAL,
                             PDLP_PRIMAL_INFEASIBLE, PDLP_DUAL_INFEASIBLE */
  int precision_used;     /* PDLP_FP64, PDLP_FP32, PDLP_USED_BF16 or PDLP_USED_PATTERN */
  int64_t iters;          /* accepted PDHG iterations */
  int64_t attempts;       /* step attempts, rejected ones included */
  int64_t restarts;
  int64_t kkt_checks;
  int64_t kernel_launches; /* kernels this call launched (setup, graph nodes, output) */
  double primal_obj, dual_obj;
  double rel_primal_res, rel_dual_res, rel_gap, rel_kkt;
  double eta, omega;      /* final step size and primal weight */
  int used_average;       /* 1 if the returned point is the weighted average iterate */
  double setup_s;         /* device setup: canonical form, transpose, scaling */
  double solve_s;         /* iteration phase, from the first step to termination */
  int lanes_A, lanes_AT;  /* lanes per row the step kernels used over A and A^T */
  double ray_obj;         /* certificate statuses: d^ (PRIMAL_INFEASIBLE) or c^T x^
                             (DUAL_INFEASIBLE); NaN otherwise */
  double ray_res;         /* the 2-norm of the certificate's residual; NaN otherwise */
  int tiles;              /* the tile step kernels that ran (pdlp_params.tiles): 0 none,
                             1 staged block tiles, 2 warp tiles */
  double upload_s;        /* batches from host buffers: the host-to-device copies of the
                             inputs (setup_s is the device setup after them); 0 otherwise */
  int persistent_form;    /* how the step attempts ran: 0 two launches per attempt,
                             1 one cooperative kernel per check period, 2 one block per
                             check period stepping from global memory, 3 one block with
                             the LP held in shared memory (persistent = 2 when the matrix,
                             vectors and iterates fit: 76 KB for a 200 x 400 relaxation
                             with 1,600 nonzeros in float64) */
  double spectral_norm;   /* halpern = 1: L, the power-iteration estimate of ||K~||_2 the
                             step size came from; 0 otherwise */
} pdlp_result;

/* Optional diagnostic outputs (same memory space as the entry point's outputs;
 * every pointer may be NULL, arrays shorter than the run are filled up to
 * their capacity):
 *  - the raw iterates at exit, unscaled and in the caller's sign convention:
 *    the current iterate (x_cur, y_cur) and the step-size-weighted average
 *    since the last restart (x_avg, y_avg);
 *  - the decision trace of the adaptive step-size rule, one entry per step
 *    attempt k = 1, 2, ...: the step size eta the attempt used, the bound
 *    eta_bar it computed (+INFINITY when dy^T K dx = 0) and whether it was
 *    accepted (1) or retried with a smaller step (0);
 *  - per KKT check: the restart taken (0 none, 1 to the current iterate, 2 to
 *    the average) and the primal weight after the check;
 *  - the current point of the last checks (unscaled, clipped to [l, u], as the
 *    check measures it): check k = 0, 1, ... writes row k mod point_capacity of
 *    check_points [point_capacity x n]; with pdlp_result.kkt_checks = K the last
 *    min(K, point_capacity) rows hold checks K - min(K, capacity) .. K - 1.  The
 *    paper suggests PDLP's cycling as a source of several reference points for
 *    fix-and-propagate (section 5; fp_run_refs).  Single LPs only.
 * The trace lets a second implementation replay the step-size sequence and
 * check every decision (the rule is sensitive enough that two correct
 * float64 implementations part after a few hundred adaptive steps). */
typedef struct {
  double* x_cur;             /* [n] */
  double* y_cur;             /* [m] */
  double* x_avg;             /* [n] */
  double* y_avg;             /* [m] */
  int64_t attempt_capacity;  /* length of eta, eta_bar, accepted */
  double* eta;
  double* eta_bar;
  int8_t* accepted;
  int64_t check_capacity;    /* length of restart, omega */
  int8_t* restart;
  double* omega;
  int64_t point_capacity;    /* rows of check_points */
  double* check_points;      /* [point_capacity x n] */
} pdlp_diagnostics;

/* Fill *p with the defaults listed above.  Returns PDLP_OK or INVALID_INPUT (p NULL). */
int pdlp_default_params(pdlp_params* p);

/* Solve eq. (1) from HOST buffers.
 *   A, b[m], sense[m], c[n], l[n], u[n]: host inputs (copied to the device).
 *   p: parameters (NULL = defaults).
 *   x0[n], y0[m]: optional warm start (NULL = cold start x = proj(0), y = 0).
 *   x_out[n], y_out[m]: host outputs (the better of the current and the
 *     average iterate at the last KKT check, by rel_kkt).
 *   r: host result struct.  diag: optional host diagnostic buffers (may be NULL).
 * Allocates and frees its own device memory; runs on a private stream and
 * returns after the result is on the host.  Uses the current CUDA device. */
int pdlp_solve(const pdlp_csr* A, const double* b, const char* sense, const double* c,
               const double* l, const double* u, const pdlp_params* p, const double* x0,
               const double* y0, double* x_out, double* y_out, pdlp_result* r,
               const pdlp_diagnostics* diag);

/* pdlp_solve whose initial primal weight comes from a hint instead of the
 * default estimate ||c~|| / ||q~|| (step A3):
 *     omega0 = ||y~_h||_2 / ||x~_h||_2,
 * the norms of the hint (x_hint[n], y_hint[m], caller's convention) after the
 * same projection and scaling a start point gets (x~ = proj(x / D_c) onto the
 * scaled bounds, y~ = proj_Y(S y / D_r)).  The primal weight balances the
 * primal and dual distances the method has to travel; when an estimate of the
 * solution is at hand, its norms give that balance (the ratio the weight
 * updates of step A10 move toward).  Used when both norms exceed 1e-10, else
 * the default; pdlp_params.fixed_omega > 0 still overrides.  The hint is
 * independent of the start (x0, y0), which may be NULL.  No counterpart in the
 * paper (which runs PDLP cold); the learned warm start (gnn.h) passes its
 * prediction here.  Returns as pdlp_solve; INVALID_INPUT if a hint is NULL. */
int pdlp_solve_hinted(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const pdlp_params* p, const double* x0,
                      const double* y0, const double* x_hint, const double* y_hint,
                      double* x_out, double* y_out, pdlp_result* r,
                      const pdlp_diagnostics* diag);

/* pdlp_time_kernels for a batch (pdlp_solve_batch's inputs, host buffers): the same
 * setup as pdlp_solve_batch, then each fused kernel over the whole batch (every LP
 * live) `reps` times from a CUDA graph; ms_per_launch[7] and bytes_per_launch[7] as in
 * pdlp_time_kernels, the bytes summed over the batch ([5] and [6] are 0: batches use
 * the two-launch form, and the whole KKT block is timed for single LPs only).  A
 * profiling aid for the batched solve below; the paper has no counterpart.  Returns
 * PDLP_OK or an error code. */
int pdlp_time_kernels_batch(int count, const pdlp_csr* const* A, const double* const* b,
                            const char* const* sense, const double* const* c,
                            const double* const* l, const double* const* u, const pdlp_params* p,
                            int reps, double* ms_per_launch, double* bytes_per_launch);

/* Primal feasibility polishing of a point x_in[n] (PDLP's feasibility polishing
 * as read here; the paper's heuristic needs LP points that satisfy the rows,
 * section 2): the PDHG of pdlp_solve on the same rows and bounds with the
 * objective replaced by 0, started from (x_in, y = 0).  A strictly feasible x_in
 * is a fixed point; a point that misses rows moves onto the feasible set, by a
 * distance of the order of its violation, the objective changing accordingly.
 * p->tol bounds the relative KKT of the objective-free problem, so the rows'
 * residual ||r_p||_2 <= tol (1 + ||b||_2).  x_out[n] (required) receives the
 * polished point, y_out[m] (may be NULL) the multipliers of the violated rows;
 * an infeasible LP ends with status PDLP_PRIMAL_INFEASIBLE and its Farkas ray.
 * Inputs, ownership and return codes as pdlp_solve. */
int pdlp_polish_primal(const pdlp_csr* A, const double* b, const char* sense, const double* l,
                       const double* u, const pdlp_params* p, const double* x_in,
                       double* x_out, double* y_out, pdlp_result* r);

/* Dual feasibility polishing of a dual point y_in[m] (the dual side of the
 * feasibility polishing above; y in the sign convention of pdlp_solve): the
 * PDHG of pdlp_solve on the dual feasibility problem -- the same rows, senses
 * and objective with b replaced by 0 and every finite bound by 0 (infinite
 * bounds stay) -- started from (x = 0, y_in).  That problem's dual has the
 * feasible set of the LP's dual and objective 0, so a dual-feasible y_in (every
 * part of lambda = c - A^T y that no finite bound carries is 0) is a fixed
 * point; otherwise y moves onto the dual feasible set by a distance of the
 * order of its violation.  p->tol bounds the relative KKT of that problem, so
 * the dual residual ||r_d||_2 <= tol (1 + ||c||_2).  y_out[m] (required when
 * m > 0) receives the polished dual point, x_out[n] (may be NULL) the
 * multipliers of the violated reduced costs; an LP whose dual is infeasible
 * ends with status PDLP_DUAL_INFEASIBLE and x_out holds its ray of descent.
 * b is not read.  Inputs, ownership and return codes as pdlp_solve (l > u in
 * any column is PDLP_ERR_INVALID_INPUT). */
int pdlp_polish_dual(const pdlp_csr* A, const char* sense, const double* c, const double* l,
                     const double* u, const pdlp_params* p, const double* y_in, double* x_out,
                     double* y_out, pdlp_result* r);

/* Solve `count` LPs of uneven size together (batched relaxations, such as those
 * left after the partial fixings of the heuristic; no counterpart in the paper).
 * Arrays of per-LP HOST pointers in the layout of pdlp_solve; one parameter
 * set for all; r[count] results.  x_out / y_out may be NULL (or hold NULL
 * entries) for outputs not wanted.
 * The LPs form one block-diagonal problem on the device: the inputs are copied to
 * their places in it, validated per LP and set up (canonical form, transpose,
 * scaling) in one pass over the whole batch -- every setup step treats each row
 * and column on its own, so each LP is set up exactly as on its own -- then every
 * step kernel and KKT pass runs over all LPs in one launch; each LP keeps its own
 * step size, primal weight, restarts and termination, and stops independently.  One CUDA
 * graph holds check_period attempts plus the KKT block of the whole batch.
 * All LPs share one precision mode: FP32_BF16A picks the pattern / bf16 form
 * only if every LP qualifies.  Limits: total rows, columns and nonzeros below
 * 2^31.  Returns PDLP_OK or an error code (an invalid LP names its index in
 * pdlp_last_error). */
int pdlp_solve_batch(int count, const pdlp_csr* const* A, const double* const* b,
                     const char* const* sense, const double* const* c, const double* const* l,
                     const double* const* u, const pdlp_params* p, double* const* x_out,
                     double* const* y_out, pdlp_result* r);

/* pdlp_solve_batch from DEVICE buffers, in stream order: A[k] are host structs whose
 * arrays are on the device, b[k] ... u[k] device pointers, x_out[k] / y_out[k] device
 * outputs (NULL entries allowed), r[count] host results, stream a cudaStream_t.  The
 * batch is validated and set up on the device as one block-diagonal problem (each LP
 * exactly as on its own: every setup step treats rows and columns one by one), with
 * one small read-back of per-LP scalars; the library allocates its scratch with the
 * stream-ordered allocator.  No counterpart in the paper.  Returns as pdlp_solve_batch. */
int pdlp_solve_batch_device(int count, const pdlp_csr* const* A, const double* const* b,
                            const char* const* sense, const double* const* c,
                            const double* const* l, const double* const* u, const pdlp_params* p,
                            double* const* x_out, double* const* y_out, pdlp_result* r,
                            void* stream);

/* Device workspace, in bytes, that pdlp_solve_device needs for this size and
 * these parameters (the precision mode decides it, and restart_metric = 1 adds
 * 16 (m + n) bytes for the gap gradients).  Returns 0 on invalid sizes.  The bound
 * holds for every value pattern. */
size_t pdlp_workspace_size(int32_t m, int32_t n, int64_t nnz, const pdlp_params* p);

/* Solve eq. (1) from DEVICE buffers, in stream order.
 *   A (struct on the host, arrays on the device), b, sense, c, l, u, x0, y0:
 *     device inputs of the same layout as pdlp_solve.
 *   x_out, y_out: device outputs.  r: HOST result struct.  diag: optional
 *     diagnostic buffers on the device (the struct itself on the host).
 *   workspace, workspace_bytes: caller-owned device scratch of at least
 *     pdlp_workspace_size(...) bytes, 256-byte aligned; NULL makes the library
 *     allocate (and free) it with the stream-ordered allocator.
 *   stream: a cudaStream_t (NULL = the legacy default stream).
 * Input validation reads the inputs back to the host once.  The call returns
 * when the solve is finished (it synchronises the stream once per KKT check
 * period to read the termination flag). */
int pdlp_solve_device(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const pdlp_params* p, const double* x0,
                      const double* y0, double* x_out, double* y_out, pdlp_result* r,
                      const pdlp_diagnostics* diag, void* workspace, size_t workspace_bytes,
                      void* stream);

/* Kernel timing for roofline reports (a profiling aid; not needed to solve).
 * Runs the same device setup as pdlp_solve_device on the same DEVICE inputs,
 * then launches each fused kernel `reps` times back to back from a CUDA graph
 * (step attempts stay live: no KKT check falls due; every timing starts from
 * the state after setup) and writes into
 * ms_per_launch[7] and bytes_per_launch[7], for
 *   [0] the primal step kernel (A^T SpMV + projected update),
 *   [1] the dual half-step (A SpMV + extrapolated update, then the step
 *       decision), timed as [2] - [0]: repeated on its own it would step y
 *       away without bound,
 *   [2] one whole attempt (the primal step, then the dual half-step),
 *   [3] the float64 KKT pass over A, [4] the float64 KKT pass over A^T,
 *   [5] one attempt inside the persistent step kernel (reps attempts in one
 *       launch; 0 when p->persistent is 0),
 *   [6] one whole KKT block as a check runs it (candidates, both passes, the
 *       decision, the restart, the flags; a reset of the check flag before each,
 *       so each block starts after a full dependency as in a solve; bytes: [3]
 *       + [4]),
 * the average device time per launch in ms (graph launch gaps included) and
 * the algorithmic bytes per launch (every array the kernel needs, each element
 * once, gathered vectors counted once).  Workspace and stream as in
 * pdlp_solve_device.  Returns PDLP_OK or an error code. */
int pdlp_time_kernels(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const pdlp_params* p, int reps,
                      double* ms_per_launch, double* bytes_per_launch, void* workspace,
                      size_t workspace_bytes, void* stream);

/* pdlp_solve_device for callers that cannot allocate device memory.
 * (No counterpart in the paper: this is a deployment variant of the solve.)
 * For code where cudaMalloc is unavailable or unwelcome -- device memory owned
 * by another allocator that must account for every byte, a latency-bound loop
 * that must not reach the CUDA driver's allocator, a caller with no workspace to
 * hand over.  Same arguments and results as pdlp_solve_device, minus the
 * workspace: the scratch is one static device array of 64 MiB inside this
 * library, which every GPU that loads the library holds until process exit.
 *  - Problems whose pdlp_workspace_size exceeds 64 MiB (67108864 bytes) are
 *    rejected with PDLP_ERR_OOM before any work.
 *  - The call makes no device allocation and creates no CUDA object (no
 *    cudaMalloc/cudaFree, pinned buffer, stream, event or graph); it launches
 *    the solver's kernels directly on `stream` and polls the termination flag
 *    in pageable host memory once per check period.
 *  - p->autotune = 1 is rejected with PDLP_ERR_INVALID_INPUT: the autotuner
 *    times its candidates with a stream, events and graphs of its own.  The
 *    size heuristic and explicit lanes_A / lanes_AT are honoured.
 *  - The first call on each device (with that device current) looks up the
 *    array's device address with cudaGetSymbolAddress and caches it.  Every
 *    call synchronises `stream` (validation, termination flag), so no call may
 *    be made while that stream is being captured.  cudaDeviceReset makes the
 *    cached address stale: do not call again on a device after resetting it.
 *  - All calls share the array, which keeps the last call's contents; every
 *    call writes what it reads, so nothing carries over, but calls whose GPU
 *    work overlaps (two streams, two host threads on one device) race on the
 *    array: serialise them per device. */
int pdlp_solve_device_noalloc(const pdlp_csr* A, const double* b, const char* sense,
                              const double* c, const double* l, const double* u,
                              const pdlp_params* p, const double* x0, const double* y0,
                              double* x_out, double* y_out, pdlp_result* r,
                              const pdlp_diagnostics* diag, void* stream);

/* ---- fix-and-propagate consumer (section 2 of the paper) --------------
 * The LP solution ranks and drives the fixings of a fix-and-propagate
 * heuristic: integers are ordered by a variable strategy (section 2, "LP-based
 * variable strategies"), fixed by LP-based randomized fixing ("LP-based
 * fixing": d_i = x - floor(x), d ~ U(0,1), floor if d > d_i else ceil), branched
 * with the integer-aware rule of Alg. 1 (2 or 3 bound changes, the fixing
 * first), propagated (linear activity bound tightening) with depth-first
 * backtracking; when every integer is fixed the remaining LP is solved (the
 * paper's "final LP", here by pdlp_solve in float64).  Host code. */
#define FP_FRAC 0     /* ascending fractionality of the LP value */
#define FP_REDCOST 1  /* descending |reduced cost| */
#define FP_DUAL 2     /* rows by descending |y|, their integers by descending |reduced cost| */
#define FP_TYPE 3     /* binaries first, then general integers (stable) */
/* Hybrid strategies (section 2, "Tiebreaking and hybrid strategies": a strategy whose
 * equally ranked variables are ordered by a second one; ties left after both keep the
 * first strategy's own tie order) */
#define FP_FRAC_DUAL 4    /* fractionality; ties by position in the FP_DUAL order */
#define FP_FRAC_REDCOST 5 /* fractionality; ties by descending |reduced cost| */
#define FP_DUAL_FRAC 6    /* FP_DUAL with each row's new integers by descending |reduced
                             cost|, then ascending fractionality; integers in no row by
                             ascending fractionality */
#define FP_REDCOST_FRAC 7 /* descending |reduced cost|; ties by ascending fractionality */
#define FP_FEASIBLE 1    /* all integers fixed and the final LP's point satisfies every
                            row to 1e-6 max(1, |b_i|) (solved at final_lp_tol; a point
                            that misses a row is polished, pdlp_polish_primal) */
#define FP_INFEASIBLE 2  /* search exhausted, root infeasible, or final LP infeasible: abort */
#define FP_NODE_LIMIT 3  /* node limit reached */
#define FP_NO_FINAL_LP 4 /* all integers fixed; final LP not requested */

typedef struct {
  size_t struct_size;  /* sizeof(fp_params); set by fp_default_params */
  int var_strategy;    /* FP_FRAC | FP_REDCOST | FP_DUAL | FP_TYPE (default) | one of the
                          hybrids FP_FRAC_DUAL .. FP_REDCOST_FRAC */
  uint64_t seed;       /* SplitMix64 seed of the fixing draws, default 1 */
  int64_t node_limit;  /* branching nodes; <= 0 means 10 x (number of integers) */
  int final_lp;        /* 1 (default): solve the final LP; 0: stop after the search */
  double final_lp_tol; /* relative KKT tolerance of the final LP, default 1e-8 */
} fp_params;

typedef struct {
  int status;              /* FP_FEASIBLE, FP_INFEASIBLE, FP_NODE_LIMIT, FP_NO_FINAL_LP */
  double obj;              /* c^T x of the returned point (NaN unless FP_FEASIBLE) */
  int64_t nodes;           /* branching nodes visited */
  int64_t backtracks;      /* exhausted nodes popped */
  int64_t final_lp_iters;  /* PDHG iterations of the final LP */
  double final_rel_primal; /* relative primal residual of the final LP */
  double search_s, lp_s;   /* host seconds in the search, in the final LP */
} fp_result;

int fp_default_params(fp_params* p);

/* Run the heuristic on HOST buffers.
 *   A, b, sense, c, l, u: the MIP's LP in the layout of pdlp_solve.
 *   x_lp[n]: an LP solution (e.g. pdlp_solve's x_out); y_lp[m]: its duals in
 *     pdlp's sign convention (needed by FP_REDCOST and FP_DUAL, else may be NULL).
 *   is_int[n]: 1 for integer columns.
 *   x_out[n]: the integer assignment (NaN in continuous columns unless the
 *     final LP ran) and, after the final LP, the whole point.
 * Returns PDLP_OK or an error code (the outcome is r->status). */
int fp_run(const pdlp_csr* A, const double* b, const char* sense, const double* c,
           const double* l, const double* u, const double* x_lp, const double* y_lp,
           const uint8_t* is_int, const fp_params* p, double* x_out, fp_result* r);

/* The heuristic from several LP reference points (the paper suggests PDLP's cycling
 * as a source of more than one reference solution, section 5; for instance the check
 * points of pdlp_diagnostics): fp_run from each x_refs[k], k < nrefs, with the same
 * y_lp, strategy and seed; the feasible result with the lowest objective is kept
 * (ties: the earlier point).  x_out and *r are that run's and *chosen its index; when
 * no run is feasible they are the last run's and *chosen is -1.  Returns PDLP_OK or an
 * error code. */
int fp_run_refs(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                const double* l, const double* u, const double* const* x_refs, int nrefs,
                const double* y_lp, const uint8_t* is_int, const fp_params* p, double* x_out,
                fp_result* r, int* chosen);

/* Name of a return code, and the last error message of the calling thread. */
const char* pdlp_error_string(int code);
const char* pdlp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PDLP_H */
