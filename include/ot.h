/*
 * ot.h - C ABI of the B300 (sm_103a) Dual (O-)BDRS optimal-transport solver.
 *
 * The library solves the unregularised discrete optimal-transport problem
 *     p* = min <C, X>  over  X >= 0, X 1 = r, X^T 1 = c          (Sec. 2, Eq. unregularized_ot_primal)
 * with the squared-Euclidean cost C_ij = kappa ||x_i - y_j||^2 between two point clouds, by the
 * log-domain Dual O-BDRS iteration of Algorithm 1 (Prop. 2; lambda = 1 is Dual BDRS, Prop. 1),
 * and certifies it with the primal-dual bounds L <= p* <= U of Proposition 3, whose upper bound is
 * evaluated as in Algorithm 2.  The cost matrix, kernel and plan are never stored: every sweep
 * recomputes C_ij in registers (linear memory, Sec. 3.2).
 *
 * Conventions (all entry points):
 *   - Every function returns ot_status and never throws or aborts.  OT_OK is success.
 *   - Inputs are borrowed for the duration of the call; outputs go to caller-owned buffers.
 *     Opaque handles are owned by the library and released by their *_destroy function.
 *   - A context, and every state created from it, may be used by one thread at a time.
 *   - Not reaching the requested tolerance is not an error: the result says why the run stopped.
 *   - A non-finite value in the iteration gives OT_ENUMERIC; the state stays readable.
 *   - A device wait that exceeds its bound gives OT_ETIMEDOUT; the state must then be recreated.
 *   - Pointers in ot_problem are host pointers unless on_device = 1, in which case they are device
 *     pointers of the context's GPU (for example the data pointers of CUDA torch tensors).
 */
#ifndef OT_B300_H
#define OT_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ot_context ot_context;
typedef struct ot_state ot_state;

typedef enum {
  OT_OK = 0,
  OT_EINVAL = 1,      /* invalid argument (sizes, weights, lambda, eps0, null pointers) */
  OT_ENOMEM = 2,      /* device or host allocation failed */
  OT_ECUDA = 3,       /* a CUDA runtime call failed (see ot_last_error) */
  OT_ENUMERIC = 4,    /* a potential or LSE became non-finite */
  OT_ETIMEDOUT = 5,   /* a bounded device wait gave up */
  OT_EBUSY = 6,       /* (serving) request not finished yet */
  OT_ECANCELLED = 7,  /* (serving) request was cancelled */
  OT_ENOTFOUND = 8    /* (serving) unknown request id */
} ot_status;

/* Arithmetic of the dual sweeps.  Certificate iterations always run compensated
 * (float-float exponent) sweeps in the FP32 modes and FP64 sweeps in OT_FP64. */
typedef enum {
  OT_EXP_MUFU = 0,    /* FP32 exponent, MUFU exp2, FP64 potentials (the fast path) */
  OT_EXP_POLY = 1,    /* FP32 exponent, exp2 by an FMA-pipe polynomial (max rel. error 5e-7) */
  OT_EXP_SPLIT = 2,   /* FP32 exponent, exp2 for a quarter of the entries by the polynomial */
  OT_FP64 = 3,        /* FP64 exponent, exp2 and sums */
  OT_FP32_COMP = 4    /* compensated float-float exponent on every iteration */
} ot_precision;

typedef enum {
  OT_STOP_TOL = 0,        /* U_best - L_best <= tol_abs or (U_best - L_best) / U_best <= tol_rel */
  OT_STOP_MAX_ITERS = 1,  /* max_iters iterations done */
  OT_STOP_TIME = 2,       /* time_budget_s exceeded (checked after each certificate) */
  OT_STOP_NONE = 3        /* ot_step: ran the requested iterations */
} ot_stop_reason;

/* Vectors of the state (Algorithm 1's return tuple and the certificate potentials). */
typedef enum {
  OT_LOG_ALPHA = 0,       /* log alpha^k              (n) */
  OT_LOG_ALPHA_HAT = 1,   /* log alpha-hat^k          (n) */
  OT_LOG_BETA = 2,        /* log beta^k               (m) */
  OT_LOG_BETA_PREV = 3,   /* log beta^{k-1}           (m) */
  OT_LOG_BETA_HAT = 4,    /* log beta-hat^k           (m) */
  OT_LOG_BETA_TILDE = 5,  /* log beta-tilde^{k-1}     (m) */
  OT_F_CERT = 6,          /* f = eps log A of the latest certificate            (n) */
  OT_G_CERT = 7,          /* g = eps log(B / c) of the latest certificate        (m) */
  OT_F_BEST = 8,          /* f of the certificate with the lowest relative gap  (n) */
  OT_G_BEST = 9           /* g of that certificate                               (m) */
} ot_vector;

/* The problem of Sec. 2: sources x (n x d, row-major) with weights a (the paper's r), targets
 * y (m x d) with weights b (the paper's c).  Weights must be finite and > 0 (or >= 0 with a
 * zero_mass_floor > 0, the paper's treatment of zero-mass pixels, App. G); they are renormalised
 * to total mass one in FP64.  d is 1, 2 or 3; n, m >= 1 and < 2^31.
 * cost_scale = kappa > 0, or 0 to use kappa = 1 / max_ij ||x_i - y_j||^2 (App. G colour cost).
 * omega >= osc(C) bounds the cost range in U = <t,w> + omega delta (Prop. 3); 0 computes
 * kappa (max - min) of the pair distances on the device. */
typedef struct {
  int64_t n, m;
  int32_t d;
  int32_t on_device;
  const float* x;
  const float* y;
  const double* a;
  const double* b;
  double cost_scale;
  double omega;
  double zero_mass_floor;
} ot_problem;

/* Algorithm 1's parameters: eps0 = eta > 0, lambda in [1, 2) (O-BDRS overrelaxation; 1 = BDRS).
 * cert_every > 0 evaluates Prop. 3 after every cert_every-th iteration; 0 never.
 * stream: a cudaStream_t to run on (0 = the context's own stream).
 *
 * Refinement (OT_EXP_MUFU only).  The FP32 exponent of the fast sweeps is a sum of terms of size
 * ~1/eps (the scaled potential and cost), so its rounding error grows as 1/eps, to about 1e-2 in
 * log2 units at eps ~ 1e-5 on a 128 x 128 grid.  There the rounding, re-injected every iteration,
 * stalls the certified gap (Prop. 3's upper bound sees it through the marginal violation delta).
 * With refinement, once the exponent's rounding bound e_fast (base 2) exceeds refine_on, each sweep
 * evaluates again in float-float (error-free transforms, as in the certificate sweeps) the chunks
 * of 16 points that hold a point's dominant terms, so that the terms left in FP32 carry at most
 * about refine_tol (natural log units) of error.  refine_on <= 0 (the default) turns refinement
 * off; refine_tol = 0 takes the default 1e-5.  A threshold of 2^-6 switches it on where, on grids,
 * the FP32 rounding starts to slow the certified gap (eps ~ 6e-5 on a 128 x 128 grid).  Its cost is
 * the float-float evaluation of every 16-point chunk that holds a dominant term of any point of a
 * warp: about 2x per late iteration on grids, more when the points' order is not spatially coherent
 * (a warp's points then have unrelated dominant targets). */
typedef struct {
  double eps0;
  double lambda;
  int64_t max_iters;
  double time_budget_s;   /* <= 0: no time budget */
  int32_t cert_every;
  int32_t precision;      /* ot_precision */
  double tol_abs;         /* <= 0: unused */
  double tol_rel;         /* <= 0: unused */
  uint64_t stream;
  int32_t algorithm;      /* ot_algorithm; 0 (OT_ALG_BDRS, Algorithm 1) unless running the ablation */
  double refine_on;       /* refinement threshold on the FP32 exponent's rounding (see above) */
  double refine_tol;      /* error the unrefined terms may carry (see above) */
} ot_params;

/* Row-update method (App. B "Annealed Sinkhorn Detailed Comparison" and App. G "Momentum and Kernel
 * Ablation"): every method shares Algorithm 1's column update, schedule and initialisation and
 * differs only in the row update.
 *   OT_ALG_BDRS         Dual (O-)BDRS (Algorithm 1): current kernel K^(lambda k + 1), momentum.
 *   OT_ALG_AS           annealed Sinkhorn: old kernel K^(k) (K^(0) = 1), no momentum.
 *   OT_ALG_AS_MOMENTUM  old kernel with the momentum extrapolation (v^{k-1})^2 / v^{k-2}.
 *   OT_ALG_AS_CURRENT   current kernel K^(k+1), no momentum.
 *   OT_ALG_DAS          debiased annealed Sinkhorn: old kernel, no momentum, numerator
 *                       (u^{k-1})^theta_k r with theta_1 = 0, theta_k = 1/k.
 * The ablation methods need lambda = 1 (the schedule eta/(k+1) they are defined on).  The
 * certificate of Prop. 3 needs the row update's kernel to be the current one (its intermediate plan
 * has row sums r only then): the old-kernel methods need cert_every = 0, and ot_certificate returns
 * OT_EINVAL for them.  The server runs OT_ALG_BDRS only. */
typedef enum {
  OT_ALG_BDRS = 0,
  OT_ALG_AS = 1,
  OT_ALG_AS_MOMENTUM = 2,
  OT_ALG_AS_CURRENT = 3,
  OT_ALG_DAS = 4
} ot_algorithm;

/* Outcome of a solve or a run of steps.  U, L are the bounds of the latest certificate,
 * U_best = min_t U_t and L_best = max_t L_t over all certificates so far (App. G.3);
 * gap_abs = U_best - L_best, gap_rel = gap_abs / U_best; best_iter is the certificate iteration
 * with the lowest relative gap (U_t - L_t) / U_t, whose potentials ot_solve returns. */
typedef struct {
  int64_t iters;
  int64_t best_iter;
  int64_t n_certs;
  double U, L, U_best, L_best, gap_abs, gap_rel;
  double eps_final;
  double elapsed_s;
  double kappa;
  double omega;
  int32_t stop;           /* ot_stop_reason */
  int32_t device_errors;  /* raw device error bits (0 when OT_OK) */
  double latency_s;       /* serving only: submission to completion (0 otherwise) */
  double queue_s;         /* serving only: submission to admission (0 otherwise) */
} ot_result;

/* Sensible defaults: eps0 = 1, lambda = 1, max_iters = 1000, cert_every = 100, OT_EXP_MUFU. */
void ot_params_default(ot_params* p);

/* Create a context on CUDA device `device` (it owns a stream and the kernel launch plans). */
ot_status ot_context_create(int device, ot_context** out);
void ot_context_destroy(ot_context* ctx);

/* Text for a status code, and the last error message recorded on a context (never NULL). */
const char* ot_status_str(ot_status s);
const char* ot_last_error(const ot_context* ctx);

/* Solve one problem with Algorithm 1 and periodic certificates until the stop rule, max_iters or
 * the time budget.  f_out (n) and g_out (m), each optional (NULL), receive the certificate
 * potentials f = eps log A, g = eps log(B/c) (Prop. 3, Eq. cert_dual_potentials) of the retained
 * iterate, host or device memory as problem->on_device says.  Allocates and frees its state. */
ot_status ot_solve(ot_context* ctx, const ot_problem* prob, const ot_params* params, double* f_out,
                   double* g_out, ot_result* res);

/* A resident solver state: Algorithm 1 initialised (log alpha^{-1} = log beta^{-1} =
 * log beta^{-2} = 0, k = 0), inputs uploaded and packed.  The problem's arrays are copied. */
ot_status ot_state_create(ot_context* ctx, const ot_problem* prob, const ot_params* params,
                          ot_state** out);
void ot_state_destroy(ot_state* st);

/* Run exactly n_iters iterations of Algorithm 1 (no stop test).  Iteration k (0-based) is a
 * certificate iteration when (k + 1) % cert_every == 0; its bounds update the result's best
 * values.  res may be NULL. */
ot_status ot_step(ot_state* st, int64_t n_iters, ot_result* res);

/* Certificate (Prop. 3 with Algorithm 2) of the last completed iteration k-1: the stored one if
 * that iteration was a certificate iteration, else a standalone compensated (or FP64) pass over
 * the state's log alpha-hat, log beta-hat, log beta-tilde.  Needs at least one iteration. */
ot_status ot_certificate(ot_state* st, ot_result* res);

/* Copy a state vector to host memory `out` (n or m doubles); *k receives the number of completed
 * iterations.  Either output may be NULL. */
ot_status ot_state_get(ot_state* st, int which, double* out, int64_t* k);

/* Resume: overwrite a state vector from host memory and set the completed-iteration count to k.
 * Only OT_LOG_ALPHA, OT_LOG_BETA and OT_LOG_BETA_PREV may be set (the inputs of iteration k);
 * the column operands of iteration k are rebuilt from them. */
ot_status ot_state_set(ot_state* st, int which, const double* in, int64_t k);

/* Tile plans (not part of the method: a tuning table).  Every instance uses the plan of its (d,
 * precision): points per thread R and chunk width CH of its sweep kernel.  The plans come from the
 * built-in table (the autotuner's choices on B300), then from tile_plans.txt beside the library
 * (written by paper_2609_33814_b300/autotune.py, read when the first context is created; the
 * environment variable OT_TILE_PLANS names another file), then from ot_set_tile_plan.  A plan applies
 * to states and server lanes created afterwards; it changes results bitwise (summation order), never
 * their accuracy.  R = 0 restores the built-in plan; OT_EINVAL for a (d, precision, R, CH) whose
 * kernel is not built (fast modes: R in {1, 2, 4} with CH in {8, 16} or R = 8 with CH = 8, the
 * polynomial modes R in {2, 4} with CH = 16; compensated: R in {1, 2, 4}, CH = 8; FP64: R in {1, 2},
 * CH = 8). */
ot_status ot_set_tile_plan(int32_t d, int32_t precision, int32_t R, int32_t ch);
ot_status ot_get_tile_plan(int32_t d, int32_t precision, int32_t* R, int32_t* ch);

/* The (kappa, omega) the state uses, after any device-side cost-range pass. */
ot_status ot_state_cost(ot_state* st, double* kappa, double* omega);

/* ---------------------------------------------------------------------------------------------
 * Output of the colour-transfer application (App. G, "Implicit implementation and output"; the
 * marginal errors of Tables 3 and 4).  For an implicit plan X = diag(u) K diag(v), K = exp(-C/eps),
 * never formed, ot_plan_project computes
 *   - the barycentric projection y_hat[i] = sum_j X_ij y_j / sum_j X_ij (n x d floats, row-major),
 *   - the row sums (n doubles) and column sums (m doubles) of X,
 *   - their errors against r and c: l1, maximum absolute, maximum relative to the prescribed mass.
 * The plan is chosen by `plan`:
 *   OT_PLAN_BEST          u = exp(f/eps), v = c exp(g/eps) from the certificate potentials f, g of
 *                         the best certificate iteration (the iterate the paper keeps); its column
 *                         sums equal c.  Needs at least one certificate, else OT_EINVAL.
 *   OT_PLAN_LATEST        u = alpha-hat, v = beta-hat of the last completed iteration.
 *   OT_PLAN_INTERMEDIATE  u = alpha-hat, v = beta-tilde of the last completed iteration: the
 *                         intermediate plan of Prop. 3, whose row sums equal r.
 * eps is that iteration's temperature (returned in err->eps).  Exponents are formed in
 * float-float and sums are Kahan-compensated FP32 (relative error of the sums ~1e-7).  Outputs are
 * host pointers, each may be NULL.  The call allocates temporary device memory (about
 * 24 (n + m) bytes plus repacked operands), waits for the state's stream, and returns OT_ENOMEM if
 * that allocation fails. */
typedef enum { OT_PLAN_BEST = 0, OT_PLAN_LATEST = 1, OT_PLAN_INTERMEDIATE = 2 } ot_plan_kind;
typedef struct {
  double row_l1, row_max_abs, row_max_rel; /* row sums against r */
  double col_l1, col_max_abs, col_max_rel; /* column sums against c */
  double eps;                              /* temperature of the plan */
} ot_marginal_errors;
ot_status ot_plan_project(ot_state* st, int32_t plan, float* y_hat, double* row_sums, double* col_sums,
                          ot_marginal_errors* err);

/* The cost of a feasible plan from an implicit one (the f of the paper's ablation, App. G "Momentum
 * and Kernel Ablation", which rounds with Altschuler, Weed and Rigollet's procedure): the rows of
 * X = diag(u) K diag(v) (plan as in ot_plan_project) are scaled down to at most r, the columns of
 * the result down to at most c, and err_r err_c^T / |err_r|_1 is added, which puts the plan in
 * Pi(r, c).  Nothing n x m is formed: three streaming passes (float-float exponents, compensated
 * sums), and the cost of the rank-one correction separates for the squared-Euclidean cost.
 * *cost_rounded = <C, rounded plan> (an upper bound on p*, valid for every ot_algorithm),
 * *cost_unrounded = <C, X>; either may be NULL.  Temporary device memory about 40 (n + m) bytes;
 * waits for the state's stream. */
ot_status ot_plan_round(ot_state* st, int32_t plan, double* cost_rounded, double* cost_unrounded);

/* ---------------------------------------------------------------------------------------------
 * Continuous-batching server.  Not in the paper: a serving front end for many independent solves
 * on one GPU.  ot_serve_submit copies the problem (host arrays, or device arrays when
 * on_device = 1) and queues it; a scheduler thread admits queued requests in arrival order into
 * free slots (max_slots) while the summed device memory of the admitted instances stays within
 * hbm_budget_bytes, and runs all admitted solves of the same d, precision and cert_every as one
 * batch: each chunk of cert_every iterations is issued as sweep launches whose work items cover
 * every instance of the batch, the last iteration of the chunk being a certificate iteration
 * for all of them.  Requests join and leave only at chunk boundaries; each stops by its own rule
 * (tol_rel / tol_abs on the best certified gap, max_iters rounded up to a multiple of
 * cert_every, time_budget_s since admission) or cancellation.  cert_every must be >= 1.
 * All ot_serve_* functions are thread-safe.  Results are the certificate potentials of the
 * retained iterate (as ot_solve), copied to host buffers f_out (n) and g_out (m), either may be
 * NULL; a finished request is released by the poll or wait call that returns it.
 * stream: a cudaStream_t for all of the server's device work (0 = a stream of its own).
 * --------------------------------------------------------------------------------------------- */
typedef struct ot_server ot_server;

typedef struct {
  int64_t submitted, completed, cancelled, failed, active, pending, chunks, launches;
  double p50_latency_s, p99_latency_s, mean_latency_s;  /* submission to completion, completed requests */
  double solves_per_s, entries_per_s, entries;          /* since creation or the last reset */
  double elapsed_s;
  double hbm_used_bytes;
} ot_serve_statistics;

ot_status ot_serve_create(ot_context* ctx, size_t hbm_budget_bytes, int32_t max_slots, uint64_t stream,
                          ot_server** out);
/* OT_ENOMEM if the request alone exceeds the budget; OT_EINVAL for invalid problems/params. */
ot_status ot_serve_submit(ot_server* sv, const ot_problem* prob, const ot_params* params, uint64_t* req_id);
/* OT_EBUSY while queued or running; otherwise the request's own status (OT_OK, OT_ECANCELLED, ...). */
ot_status ot_serve_poll(ot_server* sv, uint64_t req_id, double* f_out, double* g_out, ot_result* res);
/* Block until the request finishes or timeout_s passes (OT_EBUSY); timeout_s < 0 waits forever. */
ot_status ot_serve_wait(ot_server* sv, uint64_t req_id, double timeout_s, double* f_out, double* g_out,
                        ot_result* res);
ot_status ot_serve_cancel(ot_server* sv, uint64_t req_id);
ot_status ot_serve_stats(ot_server* sv, ot_serve_statistics* out);
/* Zero the statistics, kernel timings and launch count. */
ot_status ot_serve_reset_stats(ot_server* sv);
/* Kernel timing of the server's batched launches (as ot_profile_enable / ot_profile_read: kind 0
 * the fast iterations of a chunk, kind 1 its certificate iteration; entries = 2 n m per iteration,
 * summed over the instances a launch covers). */
ot_status ot_serve_profile_enable(ot_server* sv, int on);
ot_status ot_serve_profile_read(ot_server* sv, int kind, int64_t* launches, double* entries, double* ms);
/* The same per fast launch, in launch order: out[3 i .. 3 i + 2] = (implicit entries, milliseconds,
 * instances in the lane) for i < min(*count, max_launches); *count receives the number recorded since
 * the last reset.  out may be NULL (count only). */
ot_status ot_serve_profile_launches(ot_server* sv, double* out, int64_t max_launches, int64_t* count);
void ot_serve_destroy(ot_server* sv);

/* ---------------------------------------------------------------------------------------------
 * Allocation-free row update.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory (code running under a runtime or plugin host that owns all
 * device allocations and forbids libraries from calling cudaMalloc).  It computes
 *     log_alpha_hat[i] = log_r[i] - LSE_j( log_bt[j] - kappa ||x_i - y_j||^2 / eps )
 * with the FP32 sweep kernel of ot_step's fast iterations (its one-point-per-thread, 16-column-chunk
 * instantiation, whatever the tile plan), and allocates nothing: every buffer it
 * needs beyond its arguments lives in a fixed scratch array of about 3.2 MB inside the library,
 * which every GPU that loads the library holds until the process exits.
 *   - x (n x d floats), y (m x d floats), log_r (n doubles), log_bt (m doubles) are device inputs;
 *     log_alpha_hat (n doubles) is the device output.  1 <= n, m <= OT_NOALLOC_MAX_POINTS, d in 1..3,
 *     kappa > 0, eps > 0 (finite); anything else returns OT_EINVAL before touching the device.
 *   - stream is a cudaStream_t (0 = the legacy default stream); the call waits for it to finish.
 *   - The first call on a device looks the scratch address up for that device (with that device
 *     current) and queries the kernel's occupancy there; make that first call before any stream
 *     capture.  Later calls made outside stream capture look the address up again (this allocates
 *     nothing), so the call stays valid after the device's context is destroyed and created anew.
 *   - All calls share the one scratch array, which keeps the last call's contents (each call clears
 *     what must start at zero): calls that overlap on the GPU (from several host threads or
 *     streams) race and must not be made.
 *   - CUDA failures return OT_ECUDA; the call checks each CUDA call it makes and neither reports
 *     nor clears an error that the caller left pending.
 *   - Accuracy: log_bt enters the FP32 exponent as it is, with no gauge offset (ot_step's sweeps
 *     subtract one), so its rounding grows with max |log_bt| (about |log_bt| * 2^-24 in log2 units).
 *     A caller whose log-scalings have drifted far from zero can pass log_bt - c (c a constant, e.g.
 *     log_bt[0]): the output is then log_alpha_hat + c, so subtracting c gives log_alpha_hat for the
 *     original log_bt.
 * Returns OT_ENUMERIC if an output is non-finite. */
#define OT_NOALLOC_MAX_POINTS 16384
ot_status ot_row_update_noalloc(int64_t n, int64_t m, int32_t d, const float* x, const float* y,
                                const double* log_r, const double* log_bt, double kappa, double eps,
                                double* log_alpha_hat, uint64_t stream);

/* ---------------------------------------------------------------------------------------------
 * Row-sharded execution of one problem over `world` processes (one GPU each; the paper's solver runs
 * on one GPU, this splits Algorithm 1's sweeps for problems larger than one GPU).  Every process
 * holds the whole problem's packed operands but updates only its slice of the points of each side
 * (contiguous runs of 512 points, ot_shard_range).  One iteration is two half-sweeps: the row
 * update of the slice's rows over all columns, then the column update of its columns over all rows;
 * after each half-sweep the processes exchange the packed operands their slices rewrote (an
 * allgather of ot_shard_pack_get's bytes, applied with ot_shard_pack_put), and on certificate
 * iterations they sum the four partial sums of Prop. 3 (an allreduce of ot_shard_cert_partials):
 * L = sum rf + sum cg and U = sum <t, w> + omega sum delta.  The exchange is the caller's (for
 * example torch.distributed); no kernel waits for another process.
 *   ot_shard_range      points [*p0, *p1) of a side of np points owned by rank (no GPU needed).
 *   ot_shard_create     the slice state of `rank` (ot_state_create's arguments and conventions);
 *                       ot_step and ot_certificate refuse slice states, ot_state_get returns whole
 *                       vectors of which only the slice's entries are this process's.
 *   ot_shard_half_sweep side 0: row update of the slice, 1: column update (which completes the
 *                       iteration); cert != 0 runs the certificate iteration's sweeps (both halves
 *                       of one iteration must agree).
 *   ot_shard_pack_bytes bytes of the pack slice of `side` owned by `rank` (tiles + 8 offsets).
 *   ot_shard_pack_get   this process's pack slice of `side` into host memory.
 *   ot_shard_pack_put   another rank's pack slice of `side` from host memory (rank 0's carries the
 *                       pack offsets, which come from the first point).
 *   ot_shard_cert_partials  after a certificate column half-sweep: out[0..4] = this slice's
 *                       <r, f>, <c, g>, <t, w> (sum s_j mu_j), delta (half of sum |s_j - c_j|), and
 *                       the certificate's eps. */
ot_status ot_shard_range(int64_t np, int32_t rank, int32_t world, int64_t* p0, int64_t* p1);
ot_status ot_shard_create(ot_context* ctx, const ot_problem* prob, const ot_params* params, int32_t rank,
                          int32_t world, ot_state** out);
ot_status ot_shard_slice(ot_state* st, int32_t side, int64_t* p0, int64_t* p1);
ot_status ot_shard_half_sweep(ot_state* st, int32_t side, int32_t cert);
ot_status ot_shard_pack_bytes(ot_state* st, int32_t side, int32_t rank, size_t* bytes);
ot_status ot_shard_pack_get(ot_state* st, int32_t side, void* host_buf);
ot_status ot_shard_pack_put(ot_state* st, int32_t side, int32_t rank, const void* host_buf);
ot_status ot_shard_cert_partials(ot_state* st, double* out);

/* Measurement support (not part of the method): kernel timing.  While enabled on a context, every
 * iteration chunk of its states records CUDA events on the launching stream around its launches
 * (inside the captured CUDA graph) and waits for the chunk.  A chunk is one launch for its fast
 * iterations (row and column sweeps of every iteration) and one for its certificate iteration; per
 * kind (0 fast iterations, 1 certificate iterations) the number of launches, the algorithmic
 * implicit entries (2 n m per iteration) and the summed event durations (ms) accumulate.  Other
 * kinds return OT_EINVAL.  Any output pointer may be NULL. */
ot_status ot_profile_enable(ot_context* ctx, int on);
ot_status ot_profile_reset(ot_context* ctx);
ot_status ot_profile_read(ot_context* ctx, int kind, int64_t* launches, double* entries, double* ms);

/* Failure-injection support (tests): the number of times a sweep polls a tile's arrival before it
 * gives up, records the error and returns (the state then reports OT_ETIMEDOUT and must be
 * destroyed).  Applies to states created on this context afterwards; 0 makes every wait give up at
 * once.  The copies already in flight are still waited for, with the normal bound, before a sweep
 * returns.  The default is 2^26 polls (seconds). */
ot_status ot_debug_set_wait_limit(ot_context* ctx, uint32_t polls);

/* Test and measurement support (not part of the method): counters of a state's sweeps, into
 * out[0..8] (nout >= 9):
 *   out[0..3]  point blocks whose stored shift hint missed the sweep's exact log-sum-exp by more
 *              than 16 (base 2): row sweeps of even / odd iterations, then column sweeps of even /
 *              odd iterations, as last counted (a side's next sweep uses the hints only when the
 *              previous iteration's count of that side is 0);
 *   out[4]     warp-tiles of the fast sweeps recomputed with the exact maximum because their sum
 *              exceeded 2^64 (cumulative since the state was created);
 *   out[5..8]  micro-splits (partials per point) of the fast row and column sweeps, then of the
 *              certificate row and column sweeps;
 *   out[9]     (nout >= 10) warp-tiles of the fast sweeps whose dominant terms were evaluated again in
 *              float-float (cumulative). */
ot_status ot_state_counters(ot_state* st, int64_t* out, int32_t nout);

/* Number of CUDA kernels this context has launched since creation or the last ot_profile_reset
 * (every node of a replayed CUDA graph counts). */
ot_status ot_launch_count(ot_context* ctx, int64_t* launches);

/* Measurement support (not part of the method): pipe-throughput microbenchmarks on `device`
 * used to derive the sweep's roofline.  For probe k = 0..5 (MUFU ex2, FFMA, FFMA2, three-input
 * FMNMX, a 1 ex2 : 4 FMA : 1 FADD mix, FADD), out[2k] receives lane operations per clock per SM
 * (for the mix: exp2 per clock per SM) and out[2k+1] the SM clock in MHz seen during the probe.
 * nout >= 12; iters >= 1 sets the loop length (10^4 .. 10^5 is typical). */
ot_status ot_probe_pipes(int device, int iters, double* out, int nout);

/* exp2 of n host floats x by the fast sweep's methods, into n host floats out: method 0 the SFU's
 * ex2.approx.ftz, method 1 the FMA-pipe polynomial of OT_EXP_POLY / OT_EXP_SPLIT (x = round(x) + f,
 * a degree-5 minimax polynomial for 2^f on [-1/2, 1/2], x clamped to [-125, 126]).  Allocates and
 * frees its own device buffers on `device`; returns OT_EINVAL for other methods or n < 1. */
ot_status ot_probe_exp2(int device, int method, const float* x, float* out, int64_t n);

#ifdef __cplusplus
}
#endif

#endif /* OT_B300_H */
