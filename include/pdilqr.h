/*
 * pdilqr.h -- C ABI of the B300 primal-dual iLQR hot path.
 *
 * The library solves the linear-quadratic KKT system of each primal-dual
 * iLQR (SQP) step by the parallel associative scan of Sec. II-D of
 * "Primal-Dual iLQR for GPU-Accelerated Learning and Control in Legged
 * Robots", together with the linearisation (Sec. II-B, II-F), the FP64
 * residual and one refinement step, the parallel filter line search
 * (Sec. II-E) and the SQP loop around them.
 *
 * Conventions (Sec. II-A/II-B, with N counting control intervals and the
 * terminal cost on x_N):
 *   states x_0..x_N in R^n, controls u_0..u_{N-1} in R^m,
 *   costates lam_0..lam_N in R^n.
 * A batch holds `count` instances with a common (n, m) and horizons N_i.
 * Every per-stage array is packed instance after instance, N_i + 1 stage
 * slots per instance starting at slot stage_off[i], row-major inside a stage:
 *   A [n][n], B [n][m], c [n]      (dynamics, defect; slot N_i unused)
 *   Q [n][n], q [n]                (slot N_i holds the terminal Q_N, q_N)
 *   R [m][m], S [m][n], r [m]      (slot N_i unused; S may be NULL = 0)
 *   dx [n], du [m] (slot N_i written 0), dlam [n], K [m][n], k [m], P [n][n], p [n]
 * Unless stated otherwise every array argument is a DEVICE pointer owned by
 * the caller (for instance allocated by PyTorch) and 16-byte aligned; the
 * library never frees it.  All calls are asynchronous on the stream passed
 * (NULL = legacy default stream) and return before the GPU work ends.
 * Two calls that share a plan must not overlap on the GPU: the plan's
 * workspace is shared.  Nothing throws across this boundary; every entry
 * point returns a pdilqr_status and writes per-instance status words
 * (int32, same codes) to device memory.
 */
#ifndef PDILQR_H
#define PDILQR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PDILQR_API __attribute__((visibility("default")))
#else
#define PDILQR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pdilqr_stream; /* == cudaStream_t */

typedef enum {
    PDILQR_OK = 0,
    PDILQR_E_INVALID_ARG = 1,  /* bad size, null pointer, unsupported (n, m)      */
    PDILQR_E_NOT_SPD = 2,      /* a pivot of R_k or G_k (an SPD factorisation) was not positive */
    PDILQR_E_SINGULAR = 3,     /* a pivot of (I + C P) vanished in a combine      */
    PDILQR_E_NONFINITE = 4,    /* NaN / Inf met                                    */
    PDILQR_E_TIMEOUT = 5,      /* a bounded device or host wait ran out            */
    PDILQR_E_NO_MEMORY = 6,    /* device or pinned allocation failed               */
    PDILQR_E_ADMISSION = 7,    /* the server refused a request (memory budget)     */
    PDILQR_E_LINESEARCH = 8,   /* no step size of the grid was accepted            */
    PDILQR_E_CUDA = 9          /* a CUDA runtime call failed                       */
} pdilqr_status;

/* Static string for a status code. */
PDILQR_API const char *pdilqr_status_string(int status);

/* ------------------------------------------------------------- batches */

/* Host-side description of a batch (copied by pdilqr_plan_create).  One
 * plan serves one (n, m): the kernels are compiled per size, so a batch of
 * mixed sizes is solved through one plan per size (the server's size classes
 * do exactly that).  The problem statement of Sec. II-A/II-B fixes n and m per
 * problem; nothing in the method couples instances of different sizes. */
typedef struct {
    int32_t n;                 /* state dimension  (same for every instance)   */
    int32_t m;                 /* control dimension                             */
    int32_t count;             /* number of instances, >= 1                     */
    const int32_t *N;          /* HOST [count] horizons, 1 <= N_i <= 4096       */
    const int64_t *stage_off;  /* HOST [count] first stage slot of instance i;  */
                               /* slots [off_i, off_i + N_i] must not overlap   */
} pdilqr_batch;

typedef struct {
    int32_t warps;      /* warps per instance for the scan: 4, 8 or 16;      */
                        /* 0 picks by the longest horizon of the batch;     */
                        /* 1 runs the whole horizon in one chunk, i.e. the  */
                        /* sequential Riccati recursion inside the same     */
                        /* kernels (the comparator of the fused solver)     */
    int32_t refine;     /* 0: plain FP32 solve; 1: one refinement step      */
                        /* against the FP64-evaluated KKT residual          */
    int32_t inst_per_cta; /* instances per CTA of the batched sequential    */
                        /* SQP of one-robot SRBD problems (n = m = 12,      */
                        /* warps = 1): 2, 4 or 8 (CTAs of 1, 2 or 4 warps,  */
                        /* two instances per warp); 0 picks 2.  Other       */
                        /* solvers take one instance per CTA and require 0. */
    int32_t m_fp64;     /* 1: the scan's combines (Sec. II-D, Eq.            */
                        /* combination_rule) factor M = I + C1 P2 and apply  */
                        /* M^-1 to [A1 | C1 | b1 - C1 p2] by Gauss-Jordan   */
                        /* elimination with partial pivoting in FP64 (the    */
                        /* FP32 entries widened once, results rounded back); */
                        /* 0: in FP32.  Only (n, m) = (36, 24); other sizes  */
                        /* require 0.  The Riccati solver is unaffected.     */
    int32_t split;      /* 1: the scan's horizon chunks run on separate CTAs */
                        /* (one per chunk, warps = 8 or 16, 0 picks 16), so  */
                        /* that one instance spreads over that many SMs;    */
                        /* the CTAs of an instance meet at bounded barriers */
                        /* between the scan's phases (cooperative launch).  */
                        /* Sizes with n >= 48 only; the LQ solves           */
                        /* (pdilqr_kkt_scan_solve) and the SQP (pdilqr_solve,*/
                        /* then unfused) use it.  Errors: INVALID_ARG for   */
                        /* other sizes or warps; a launch whose warps x     */
                        /* count CTAs cannot all be resident fails (CUDA).  */
} pdilqr_opts;

typedef struct pdilqr_plan pdilqr_plan;

/* Validate a batch, copy its description to the current CUDA device and
 * allocate the plan's workspace (device memory, about (2n^2 + nm + 3n + m)
 * floats per stage slot).  Supported (n, m): (1,1) (2,1) (3,2) (4,2),
 * (36,24) (the whole-body-sized LQ problem), and the SRBD sizes
 * (12 R, 12 R) for R = 1, 2, 4, 8, 16 robots, which also have the
 * linearisation, the merit and the fused SQP.  Every size has both the scan
 * and the Riccati solvers.  Errors: INVALID_ARG, NO_MEMORY, CUDA.  *out is
 * NULL on error. */
PDILQR_API pdilqr_status pdilqr_plan_create(const pdilqr_batch *batch, const pdilqr_opts *opts,
                                 pdilqr_plan **out);
PDILQR_API pdilqr_status pdilqr_plan_destroy(pdilqr_plan *plan);
/* Warps per instance the plan uses for the scan (after the 0 -> pick rule). */
PDILQR_API int32_t pdilqr_plan_warps(const pdilqr_plan *plan);

/* Test switches of a plan (0 = none, the default).  They exist to exercise
 * failure handling without faulting the GPU and are never needed otherwise.
 *   PDILQR_DEBUG_TC_SKIP_ISSUE: the tensor-core products (one-chunk kernels of
 *   n >= 96) issue neither their MMAs nor the commit that signals them, so the
 *   bounded wait for them runs out (after about 0.6 s per CTA); the instance
 *   then ends with status PDILQR_E_TIMEOUT and the context stays usable.
 *   PDILQR_DEBUG_BULK_SKIP_ISSUE: the one-CTA Riccati recursion of n = 24 and 36
 *   (pdilqr_riccati_solve) issues none of its bulk stage copies, so the
 *   bounded wait for the first one runs out (about 0.6 s per CTA); the
 *   instance ends with status PDILQR_E_TIMEOUT and the context stays usable.
 *   PDILQR_DEBUG_SPLIT_SKIP_ARRIVE: in the split scan (pdilqr_opts.split) the
 *   CTA of chunk 0 does not arrive at the first barrier between the scan's
 *   phases, so the bounded wait of every CTA of the instance runs out (about
 *   2 s); the instance ends with PDILQR_E_TIMEOUT (its results are not
 *   meaningful) and the context stays usable.
 * Errors: INVALID_ARG (unknown bits). */
#define PDILQR_DEBUG_TC_SKIP_ISSUE 1
#define PDILQR_DEBUG_BULK_SKIP_ISSUE 2
#define PDILQR_DEBUG_SPLIT_SKIP_ARRIVE 4
PDILQR_API pdilqr_status pdilqr_plan_set_debug(pdilqr_plan *plan, int32_t flags);

/* ------------------------------------------------------- LQ KKT solves */

/* LQ data of a batch (device, layout above).  In Sec. II-B notation: A, B the
 * dynamics Jacobians, c the defects b_i, Q, R, S the Hessian blocks, q, r the
 * Lagrangian gradients; slot N_i of Q, q is the terminal P_{N+1}, p_{N+1}. */
typedef struct {
    const float *A, *B, *c, *Q, *R, *S, *q, *r;
} pdilqr_lq;

typedef struct {
    float *dx, *du, *dlam;     /* required outputs (search direction, Eq. QP)   */
    float *K, *k, *P, *p;      /* optional outputs (NULL: kept in the plan)     */
    int32_t *status;           /* required [count] per-instance status          */
    double *resid;             /* optional [count][4]: infinity norms of the    */
                               /* final KKT residual, of the KKT matrix (max    */
                               /* absolute row sum), of z and of the right-hand */
                               /* side; backward error = r0 / (r1 r2 + r3)      */
} pdilqr_kkt_out;

/* LQ KKT solve by the parallel associative scan (Sec. II-D): conditional
 * value function elements (Eq. initialization) combined by the combination
 * rule (corrected as documented in kkt_scan.cuh) in a chunked reduce-then-scan
 * over the horizon, parallel policy recovery (Eq. lqr), the trajectory scan
 * of Eq. (controlled_dynamics) and dlam_i = P_i dx_i + p_i.  s [count][n] is
 * dx_0 = xhat_0 - x_0.  With opts.refine the KKT residual is evaluated in FP64
 * and one correction solve is added.  One CTA per instance. */
PDILQR_API pdilqr_status pdilqr_kkt_scan_solve(pdilqr_plan *plan, const pdilqr_lq *lq, const float *s,
                                    pdilqr_kkt_out *out, pdilqr_stream stream);

/* The same system by the sequential Riccati recursion and forward rollout of
 * Sec. II-C (the comparator): one warp per instance for n <= 12, one CTA of
 * 128 threads per instance for (n, m) = (24, 24) and (36, 24), with the
 * larger sizes again one warp per instance; honours opts.refine.  Status per
 * instance as for pdilqr_kkt_scan_solve (E_NOT_SPD when a pivot of some
 * G_k = R_k + B_k^T P_k+1 B_k is not positive, E_NONFINITE when an output is
 * not finite). */
PDILQR_API pdilqr_status pdilqr_riccati_solve(pdilqr_plan *plan, const pdilqr_lq *lq, const float *s,
                                   pdilqr_kkt_out *out, pdilqr_stream stream);

/* FP64 evaluation of the KKT residual of z = (dx, du, dlam); writes the four
 * norms described under pdilqr_kkt_out.resid to resid [count][4] (device). */
PDILQR_API pdilqr_status pdilqr_kkt_residual(pdilqr_plan *plan, const pdilqr_lq *lq, const float *s,
                                  const float *dx, const float *du, const float *dlam,
                                  double *resid, pdilqr_stream stream);

/* --------------------------------------------- allocation-free scan solve */

/* The LQ KKT scan solve of pdilqr_kkt_scan_solve for callers that may not
 * allocate device memory at all -- a real-time control loop whose timing
 * budget cannot absorb cudaMalloc (it can block and synchronise the device),
 * code running while a CUDA graph is being captured (where cudaMalloc is not
 * allowed), or a host application whose memory pool already owns the GPU.
 * The paper has no counterpart: this is an interface of this library only.
 *
 * No plan is used and nothing is allocated: the per-stage workspace (policy,
 * value function, closed-loop maps) lives in one static device array of
 * 16 MiB that every GPU loading the library holds until the process exits.
 * The caller passes inputs and outputs as in pdilqr_kkt_scan_solve, plus the
 * batch tables as DEVICE arrays N [count] and stage_off [count] and the
 * number of stage slots total_stages (>= max(stage_off + N + 1)); warps is
 * 4, 8, 16 or 0 (= 8).  The instances' slot ranges [stage_off_i,
 * stage_off_i + N_i] must be disjoint, as for pdilqr_kkt_scan_solve: they
 * live in device memory, so this call cannot check it, and overlapping
 * ranges race on the scratch and on dx, du, dlam.  Batches needing more than
 * pdilqr_noalloc_capacity_stages(n, m) stage slots are rejected with
 * PDILQR_E_INVALID_ARG before any GPU work; an instance whose slots fall
 * outside total_stages gets status PDILQR_E_INVALID_ARG and is skipped.  No
 * refinement step.  The first call on a device looks up the array's device
 * address (once per device); make that first call before any stream
 * capture.  Every call shares the array: calls that overlap on the GPU race
 * and must be serialised by the caller (one stream, or events).  No part of
 * the array needs clearing between calls: every workspace slot a solve reads
 * was written earlier in the same solve. */
PDILQR_API pdilqr_status pdilqr_kkt_scan_solve_noalloc(
    int32_t n, int32_t m, int32_t count, int64_t total_stages, const int32_t *N,
    const int64_t *stage_off, int32_t warps, const pdilqr_lq *lq, const float *s, float *dx,
    float *du, float *dlam, int32_t *status, pdilqr_stream stream);

/* Stage slots that the static array holds for state / control sizes (n, m). */
PDILQR_API int64_t pdilqr_noalloc_capacity_stages(int32_t n, int32_t m);

/* ------------------------------------------------------ SRBD model, Sec. III */

/* Single-rigid-body quadruped (the paper prints no equations; this is the
 * library's reading).  Per robot x = [p, theta, v, omega] (n = 12) and
 * u = [f_0..f_3] ground reaction forces (m = 12); with stance flags s_j:
 *   p' = v,  theta' = omega,  v' = sum_j s_j f_j / mass - g e_z,
 *   omega' = I^-1 ( sum_j s_j (foot_j - p) x f_j - omega x (I omega) ),
 * one explicit Euler step of length dt.  Stage cost (Sec. II-F):
 *   0.5 |x - xref|_W^2 + 0.5 |u - uref|_Wu^2 + sum over stance feet of the
 *   relaxed barrier B(xi; bar_mu, bar_delta) of the five friction-pyramid rows
 *   xi = mu f_z +- f_x, mu f_z +- f_y, f_z;
 * terminal cost 0.5 |x_N - xref_N|_WN^2.  With nrob > 1 robots are stacked
 * (n = m = 12 nrob) and a ring formation cost
 * 0.5 w_form sum_a |p_a - p_{a+1 mod nrob} - d_form[a]|^2 is added at every
 * stage.  The Hessian is the Gauss-Newton one of Sec. II-F. */
typedef struct {
    int32_t nrob;              /* robots stacked in one state: 1, 2, 4, 8, 16   */
    float w_form;              /* formation weight                              */
    float d_form[16][3];       /* formation offsets                             */
    float mass, inertia[3], dt, gravity;
    float foot[4][3];          /* stance points, world frame                    */
    float mu_fric, bar_mu, bar_delta;
    float W[12], Wu[12], WN[12];   /* diagonal weights of one robot             */
} pdilqr_srbd_model;

/* Trajectory of a batch (device, N_i + 1 slots per instance):
 * x, lam [n], u [m] (slot N_i unused), xref [n], uref [m],
 * contact [nrob][4] uint8 stance flags, x0hat [count][n]. */
typedef struct {
    const float *x, *u, *lam, *xref, *uref;
    const uint8_t *contact;
} pdilqr_traj;

/* Mutable LQ data (outputs of pdilqr_linearize), same layout as pdilqr_lq. */
typedef struct {
    float *A, *B, *c, *Q, *R, *S, *q, *r;
} pdilqr_lq_out;

/* Linearisation of Sec. II-B/II-F for every stage in parallel: A = dh/dx,
 * B = dh/du, c_k = h(x_k, u_k) - x_{k+1}, Gauss-Newton Q, R (barrier
 * curvature included), S = 0 (written if non-NULL), q = grad_x l + A^T
 * lam_{k+1} - lam_k, r = grad_u l + B^T lam_{k+1}; slot N: Q_N, q_N =
 * grad l_N - lam_N.  One warp per stage slot.  Needs n = m = 12 nrob. */
PDILQR_API pdilqr_status pdilqr_linearize(pdilqr_plan *plan, const pdilqr_srbd_model *model,
                                          const pdilqr_traj *traj, pdilqr_lq_out *out,
                                          pdilqr_stream stream);

/* Line-search merit of Sec. II-E for the ten step sizes alpha_t = 2^-t,
 * t = 0..9, per instance: merit[count][24] (device, double) receives
 *   [0] J(0)   [1] theta(0)   [2] dphi = grad J^T dz
 *   [3 + t]  J(alpha_t) - J(0)   [13 + t] theta(alpha_t)   [23] unused,
 * where theta = |xhat_0 - x_0|_2 + sum_k |x_{k+1} - h(x_k, u_k)|_2 and the
 * cost differences are evaluated stage by stage in a cancellation-free form.
 * dz = (dx, du) is the search direction (device, trajectory layout). */
PDILQR_API pdilqr_status pdilqr_merit_eval(pdilqr_plan *plan, const pdilqr_srbd_model *model,
                                           const pdilqr_traj *traj, const float *x0hat,
                                           const float *dx, const float *du, double *merit,
                                           pdilqr_stream stream);

/* SQP options (Sec. II-E).  theta_max = theta_frac * max(1, theta(initial
 * iterate)); above it a step must lower theta; below it a descent direction
 * must satisfy Armijo J(a) <= J(0) + c_armijo a dphi with theta(a) <= theta_max,
 * otherwise the cost or theta must drop.  The largest accepted step of the
 * grid 2^0..2^-9 is taken. */
typedef struct {
    int32_t max_iters;         /* SQP iterations, 1..32                          */
    float tol_step;            /* stop when |dz|_inf < tol_step and             */
    float tol_theta;           /*   theta < tol_theta (0 never stops early)     */
    float c_armijo;            /* Armijo constant (1e-4)                         */
    float theta_frac;          /* theta_max fraction (1e-2)                      */
    const float *alpha_replay; /* device [count][max_iters] step sizes to use    */
                               /* instead of the line search, or NULL           */
} pdilqr_sqp_opts;

typedef struct {
    int32_t *iters;            /* [count] KKT solves performed                   */
    int32_t *status;           /* [count] OK, LINESEARCH, NOT_SPD, SINGULAR      */
    float *alpha;              /* [count][max_iters] steps taken (optional)      */
    double *J, *theta;         /* [count] merit at the returned iterate (opt.)   */
} pdilqr_sqp_info;

/* Full multiple-shooting SQP (Sec. II-B..II-E) on the SRBD model: per
 * iteration the linearisation, the LQ KKT solve by the parallel scan, the
 * parallel line search over the ten step sizes and the update
 * x += a dx, u += a du, lam += a dlam (Eq. linear_rollout), all in one
 * kernel with one CTA per instance and no host synchronisation.  x, u, lam
 * (device, trajectory layout) hold the warm start on entry and the solution
 * on exit.  Needs n = m = 12 nrob with nrob in {1, 2, 4, 8, 16}.  Sizes
 * whose work areas exceed shared memory (nrob >= 8) run them from a global
 * workspace the plan allocates.  A split plan (pdilqr_opts.split, nrob >= 4)
 * runs each iteration unfused instead, all on the stream: the linearisation
 * of every stage into the plan's LQ arrays, the scan with its chunks on
 * separate CTAs, and one kernel per iteration for the merit of the ten step
 * sizes, the filter decision and the update (the same rules as the fused
 * kernel); such plans cannot be captured (pdilqr_solve_capture refuses
 * them). */
PDILQR_API pdilqr_status pdilqr_solve(pdilqr_plan *plan, const pdilqr_srbd_model *model,
                                      const pdilqr_sqp_opts *opts, const float *x0hat,
                                      float *x, float *u, float *lam, const float *xref,
                                      const float *uref, const uint8_t *contact,
                                      pdilqr_sqp_info *info, pdilqr_stream stream);

/* Capture one pdilqr_solve with these arguments into a CUDA graph that the
 * plan owns (replacing the plan's earlier graph, if any); pdilqr_plan_replay
 * then launches it.  The graph holds the arguments' device pointers and the
 * option values as they are now: a replay solves in place on the same
 * arrays (x, u, lam are read as the warm start and overwritten, the info
 * arrays rewritten), so the caller refills the inputs between replays.
 * Nothing runs on the GPU during the capture.  The capture uses a private
 * stream in relaxed mode; it may not be called while the calling thread
 * captures another stream.  Errors: as pdilqr_solve, CUDA; INVALID_ARG for a
 * split plan. */
PDILQR_API pdilqr_status pdilqr_solve_capture(pdilqr_plan *plan, const pdilqr_srbd_model *model,
                                              const pdilqr_sqp_opts *opts, const float *x0hat,
                                              float *x, float *u, float *lam, const float *xref,
                                              const float *uref, const uint8_t *contact,
                                              pdilqr_sqp_info *info);
/* Launch the plan's captured solve on `stream` (asynchronous).  Errors:
 * INVALID_ARG (no graph captured), CUDA. */
PDILQR_API pdilqr_status pdilqr_plan_replay(pdilqr_plan *plan, pdilqr_stream stream);

/* ------------------------------------------------------------ serving loop */

/* A continuous-batching MPC server (the real-time iteration of Sec. II-F: one
 * SQP iteration per control tick, warm-started from the previous solution
 * shifted by one step).  Clients submit requests from host memory at any
 * time; a dispatcher thread admits them into device slots, batches the
 * requests whose clients are idle (grouped by state size), launches the fused
 * SQP on one of several streams while other batches are still running, and
 * completes tickets as their batch finishes.  Warm-start trajectories,
 * multipliers and references stay resident on the device per client.
 * Admission: a client's state is carved from a device pool of
 * hbm_budget_bytes, and the first client of a size class is admitted only if
 * the device's free memory (cudaMemGetInfo) holds that class's batch
 * workspace for every stream that may run it plus hbm_reserve_bytes; when
 * either does not fit the submit fails with PDILQR_E_ADMISSION.  All waits
 * are bounded. */
typedef struct {
    int64_t hbm_budget_bytes;  /* device pool for client state (0: 1 GiB)         */
    int32_t max_batch;         /* requests per launch (0: 1024; 1: one per launch);
                                  a class of 2^c robots takes at most
                                  max(64, max_batch / 4^c), never above max_batch */
    int32_t max_inflight;      /* batches in flight on separate streams, 1..16
                                  (0: 2); classes of 4+ robots hold at most all
                                  but one */
    int32_t max_N;             /* longest horizon a client may use (0: 100)       */
    int32_t sqp_iters;         /* SQP iterations per request (0: 1)               */
    int32_t warps;             /* horizon chunks per instance, an upper bound    */
                               /* (0: 8; 1: sequential Riccati); a size class   */
                               /* runs the largest count whose fused kernel     */
                               /* fits shared memory, else 1                     */
    int32_t batch_window_us;   /* how long the dispatcher waits for more requests */
                               /* once it has one and a stream is free (0: none)  */
    pdilqr_srbd_model model;   /* robot and formation constants (shared by all    */
                               /* clients); nrob is taken per client              */
    const pdilqr_srbd_model *class_models;  /* HOST [5] or NULL: the constants of */
                               /* the classes nrob = 1, 2, 4, 8, 16 (their nrob    */
                               /* fields are ignored; read during create only);    */
                               /* NULL: `model` for every class                    */
    int64_t hbm_reserve_bytes; /* device memory left free when a size class's     */
                               /* batch workspace is first needed (0: 256 MiB)    */
    int32_t large_cta_budget;  /* most instances of the classes of 4+ robots in   */
                               /* flight at once (each runs on one CTA for tens  */
                               /* of milliseconds); a large batch is launched    */
                               /* only while the budget has room and is cut to   */
                               /* it, so that the SMs it leaves serve the small  */
                               /* classes.  0: no budget (streams limit alone)   */
    int32_t split_min_robots;  /* classes of at least this many robots (4, 8 or   */
                               /* 16) run split plans: the scan's 16 horizon     */
                               /* chunks of an instance on 16 CTAs, an unfused   */
                               /* SQP iteration (as pdilqr_opts.split); at most  */
                               /* one split batch is in flight.  0: none (every  */
                               /* class runs the fused kernel)                   */
    int32_t split_max_batch;   /* most instances of one split batch (0: 8; each   */
                               /* holds 16 SMs while it runs); with split classes */
                               /* 16 x split_max_batch above the device's SM     */
                               /* count is an invalid argument                   */
} pdilqr_serve_opts;

typedef struct {
    int32_t nrob;              /* robots of this client: 1, 2, 4, 8 or 16        */
                               /* (n = m = 12 nrob); fixed                        */
    int32_t N;                 /* horizon of this client; fixed                   */
    int32_t reset;             /* 1: re-initialise the warm start from x0hat      */
    const float *x0hat;        /* HOST [n] measured state                         */
    const float *xref;         /* HOST [N+1][n] or NULL (keep, shifted one step)  */
    const float *uref;         /* HOST [N+1][m] or NULL (required with xref)      */
    const uint8_t *contact;    /* HOST [N+1][nrob][4] or NULL (required with xref)*/
} pdilqr_request;

typedef struct {
    int32_t status;            /* status of the solve                             */
    int32_t iters;             /* SQP iterations run                              */
    int64_t latency_ns;        /* submit to completion                            */
    float *u0;                 /* caller's HOST [m] buffer for u_0, or NULL       */
    float *x, *u;              /* caller's HOST [N+1][n], [N+1][m] buffers, or NULL */
} pdilqr_result;

typedef struct {
    int64_t submitted, completed, refused, batches;
    int64_t clients, pool_bytes_used, pool_bytes_total;
    double mean_batch, p50_latency_us, p99_latency_us, solves_per_s;
} pdilqr_serve_stats_t;

typedef struct pdilqr_server pdilqr_server;

/* Create a server on the current CUDA device (the pool is allocated here). */
PDILQR_API pdilqr_status pdilqr_serve_create(const pdilqr_serve_opts *opts, pdilqr_server **out);
/* Queue a request of client `client_id` (host data copied before return).  A
 * new client is admitted here and must pass xref, uref and contact. */
PDILQR_API pdilqr_status pdilqr_serve_submit(pdilqr_server *srv, uint64_t client_id,
                                             const pdilqr_request *req, uint64_t *ticket);
/* Wait up to timeout_us for a ticket; on success the ticket is consumed and
 * the result copied to the caller's buffers; PDILQR_E_TIMEOUT otherwise. */
PDILQR_API pdilqr_status pdilqr_serve_poll(pdilqr_server *srv, uint64_t ticket,
                                           pdilqr_result *res, int64_t timeout_us);
/* Free a client's device state (fails while it has a request in flight). */
PDILQR_API pdilqr_status pdilqr_serve_release(pdilqr_server *srv, uint64_t client_id);
/* Copy a client's warm start (x, u, lam in the trajectory layout, HOST) out,
 * or back in; used to checkpoint and resume a controller. */
PDILQR_API pdilqr_status pdilqr_serve_snapshot(pdilqr_server *srv, uint64_t client_id, float *x,
                                               float *u, float *lam);
PDILQR_API pdilqr_status pdilqr_serve_restore(pdilqr_server *srv, uint64_t client_id,
                                              const float *x, const float *u, const float *lam);
PDILQR_API pdilqr_status pdilqr_serve_stats(pdilqr_server *srv, pdilqr_serve_stats_t *out);
/* Finish in-flight batches (bounded wait), free everything. */
PDILQR_API pdilqr_status pdilqr_serve_destroy(pdilqr_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* PDILQR_H */
