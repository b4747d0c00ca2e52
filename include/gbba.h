/*
 * gbba.h -- C ABI of the GB300 bundle-adjustment hot path (libgbba.so).
 *
 * Levenberg-Marquardt with a matrix-free, block-Jacobi-preconditioned conjugate
 * gradient on the damped normal equations (PCGNR), for the Snavely reprojection
 * factor of arXiv 2605.30583 (Caspar), Sec. V and Sec. VI-A.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns a ba_status; BA_OK is 0.  On failure ba_last_error()
 *    returns a message for the calling thread.  No call aborts the process.
 *  - Cameras are 9 doubles each, in this order: rotation vector w (3),
 *    translation t (3), focal length f, radial terms k1, k2.  Points are 3
 *    doubles.  Both are row-major arrays ("user layout"): cams[n_cams][9],
 *    pts[n_pts][3].  Pixels are pixels[n_obs][2].
 *  - The camera model is P = R(w) X + t, p = -P.xy / d_safe with
 *    d_safe = P.z + eps_depth * sign_no_zero(P.z), pixel = f (1 + k1|p|^2 +
 *    k2|p|^4) p, residual = pixel - measured (Sec. VI-A).
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global
 *    memory of the current device.  Pointers are borrowed: the library never
 *    frees caller memory and keeps no caller pointer beyond the call, except the
 *    workspace and stream given to ba_bind_workspace.
 *  - All device memory the library uses lives in ONE caller-allocated workspace
 *    (Sec. V-A: a single allocation for the whole optimisation, arrays are views
 *    into it).  The library itself calls no cudaMalloc.
 *  - Device work is enqueued on the stream given to ba_bind_workspace.  Calls
 *    that return host data synchronise that stream.
 *  - One problem may be used by one host thread at a time.
 */
#ifndef GBBA_H
#define GBBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BA_OK = 0,
    BA_ERR_INVALID_ARG = 1,          /* bad size, index, pointer or option          */
    BA_ERR_CUDA = 2,                 /* a CUDA runtime call failed                  */
    BA_ERR_WORKSPACE_TOO_SMALL = 3,  /* bound workspace smaller than ba_workspace_size */
    BA_ERR_NUMERIC = 4,              /* NaN/Inf, or a preconditioner block not SPD  */
    BA_ERR_TIMEOUT = 5,              /* a bounded device wait ran out               */
    BA_ERR_NOT_IMPLEMENTED = 6,
    BA_ERR_STATE = 7                 /* call made in the wrong order (e.g. no workspace) */
} ba_status;

typedef enum {
    BA_PREC_MIXED = 0,   /* FP32 Jacobians, operator and PCG vectors; FP64 master
                            parameters (the kernels read their FP32 rounding);
                            double-float residuals (ba_options.residual_precision);
                            FP64 cost sums, PCG dot products and block inversions */
    BA_PREC_FP64 = 1     /* plain all-FP64 form: stored FP64 Jacobian, FP64 vectors,
                            per-observation atomics (the comparison baseline)      */
} ba_precision;

typedef struct ba_problem ba_problem;

/* Solver options.  Defaults (ba_options_default) follow Sec. VI of the paper:
 * initial trust region 100 (mu_0 = 1/100) and CG tolerance 1e-3. */
typedef struct {
    int32_t max_lm_iters;         /* LM iterations (accepted or rejected), default 20   */
    int32_t max_pcg_iters;        /* PCG iterations per LM iteration, default 50        */
    double pcg_rel_tol;           /* stop when |r_k|_2 <= tol |r_0|_2, default 1e-3     */
    double initial_trust_region;  /* mu_0 = 1 / initial_trust_region, default 100       */
    double min_diag;              /* D = clamp(diag(J^T J), min_diag, max_diag)         */
    double max_diag;
    double max_mu;                /* stop when mu exceeds this, default 1e16 (a step is
                                     then ~1e-16 of the gradient step: below the
                                     parameters' resolution).  The mixed form caps it at
                                     1e16: beyond that its FP32 PCG products underflow */
    double eps_depth;             /* epsilon of d_safe (Sec. VI-A), default 0           */
    int32_t use_graph;            /* 1 (default): one CUDA graph; its LM and PCG loops are
                                     device-driven conditional nodes, except with the
                                     persistent PCG kernel, where the graph holds the
                                     fixed LM sequence (as for 2);
                                     2: one graph of the fixed sequence of max_lm_iters x
                                     max_pcg_iters slots, idle slots return at once;
                                     0: the same sequence launched from the host    */
    int32_t pcg_kernel;           /* 2 (default): one persistent cooperative kernel per PCG
                                     solve when every CTA's tiles fit in shared memory,
                                     with the recurrences arranged so that one grid-wide
                                     exchange per iteration carries both inner products,
                                     and residual replacement: when the recursively
                                     updated residual meets the tolerance, the true
                                     residual b - A h is computed and the recurrences
                                     restart from it, so the solve stops on a true
                                     residual (at most 4 checks per solve); where its
                                     plan does not fit but the two-exchange one does
                                     (it holds private camera copies), the latter;
                                     0: the persistent kernel with the textbook
                                     recurrences (two exchanges per iteration);
                                     1: separate kernels per PCG iteration (also used
                                     when the persistent plan does not fit);
                                     3: separate kernels per PCG iteration with the
                                     one-reduction recurrences: each iteration's update
                                     is fused into the next operator application (falls
                                     back to 1 when a tile's observations exceed the
                                     tile kernels' shared-memory stage)             */
    int32_t rotation_update;      /* how a step updates each camera's rotation:
                                     0 (default): additive angle-axis, w <- w + dw, the
                                     Jacobian taken w.r.t. w (through the left Jacobian
                                     J_l(w) of the exponential map);
                                     1: tangent-space retraction (the paper's Pose3
                                     update, Sec. VI-A), R <- Exp(d) R(w), the Jacobian
                                     taken w.r.t. d at d = 0, and w <- Log(Exp(d) Exp(w))
                                     stored back in angle-axis form.  ba_evaluate, the
                                     autograd entries and ba_cost_noalloc always use w. */
    int32_t loss;                 /* robust loss on s = |r_o|^2 of each observation, F =
                                     1/2 sum rho(s): 0 squared (default, rho = s);
                                     1 Huber (rho = s for s <= d^2, else 2 d sqrt(s) - d^2);
                                     2 Cauchy (rho = d^2 log(1 + s/d^2)).  LM runs on the
                                     IRLS-weighted system J^T W J + mu D, W = rho'(s) at
                                     the linearisation point.  Not in the batched mode.  */
    double loss_scale;            /* the loss's scale d in pixels, default 1              */
    int32_t solver;               /* 0 (default): PCGNR on the full damped normal
                                     equations (Sec. V); 1: PCG on the camera Schur
                                     complement S = H'cc - Hcp H'pp^-1 Hpc with the points
                                     back-substituted (the alternative Sec. V sets aside),
                                     block-Jacobi on the camera blocks.  Mixed precision
                                     only (BA_ERR_NOT_IMPLEMENTED for the FP64 form and
                                     the batched mode).                                 */
    int32_t wait_timeout_ms;      /* limit on each grid-wide wait of the persistent PCG
                                     kernel (its CTAs meet at a barrier twice per
                                     iteration), default 2000.  A wait that does not end
                                     within it gives up: every CTA leaves the kernel and
                                     the solve reports BA_ERR_TIMEOUT (the context stays
                                     usable).  0 gives up at the first poll that finds
                                     the barrier incomplete.  0..60000.  The separate-
                                     kernel PCG and the batched mode have no grid-wide
                                     waits and ignore it.                              */
    int32_t residual_precision;   /* arithmetic of the mixed form's residuals r = f s p - u
                                     (the cost LM minimises and the r of g = J^T r):
                                     1 (default): double-float (pairs of FP32 values,
                                     ~48 bits) from FP64 master parameters, then rounded
                                     to FP32, so r carries ~1e-7 px of error instead of
                                     FP32's ~1e-4 px, which LM can otherwise exploit
                                     along poorly constrained directions; 0: FP32.  The
                                     Jacobian, the normal operator and PCG are FP32
                                     either way; the FP64 form and the batched mode
                                     ignore it.                                         */
} ba_options;

/* One LM iteration (Sec. V): cost before the step, candidate cost, damping used,
 * gain ratio, PCG iterations spent, whether the step was accepted, and the device
 * time (ns since the start of the solve) at which the decision was taken. */
typedef struct {
    double cost;
    double cost_new;
    double mu;
    double rho;
    double model_decrease;
    int32_t pcg_iters;
    int32_t accepted;
    int64_t t_ns;
} ba_iter_stat;

typedef struct {
    double initial_cost;
    double final_cost;
    int32_t lm_iters;
    int32_t accepted;
    int32_t pcg_iters_total;
    int32_t status;               /* ba_status of the device-side solve            */
    int64_t solve_ns;             /* device time of the whole solve                */
} ba_stats;

const char* ba_last_error(void);
const char* ba_status_string(int32_t status);
/* Version of the structs above: 2 since ba_options gained wait_timeout_ms and
 * residual_precision (a caller built against version 1 passes a shorter struct). */
int32_t ba_abi_version(void);

/* Self-test of the bounded grid waits that every cooperative kernel of this library
 * uses (the persistent PCG kernel's barriers).  Launches a cooperative grid of `grid`
 * CTAs (1 <= grid <= the SM count) that waits at a barrier counting one CTA more than
 * it has, which nothing completes; each CTA must give up after timeout_ms (1..2000)
 * and return, leaving the context usable.  scratch: 16 bytes of caller-owned device
 * memory, 16-byte aligned.  On BA_OK, *gave_up is the number of CTAs that gave up
 * (grid when the mechanism works) and *error_word the shared error flag (1).  No GPU
 * fault is involved: the wait simply runs out. */
ba_status ba_selftest_wait_timeout(void* scratch, int32_t grid, int32_t timeout_ms, void* stream, int32_t* gave_up,
                                   int32_t* error_word);

/* Self-test of the FP64 reciprocal that the block-Jacobi inversions use (a hardware
 * approximation refined by two Newton-Raphson steps).  y[i] = 1/x[i] for i < n, with
 * x and y device arrays of n doubles (n >= 1), enqueued on `stream` (cudaStream_t).
 * Zero, non-finite and |x| outside [1e-300, 1e300] take the IEEE quotient 1.0 / x. */
ba_status ba_selftest_rcp64(const double* x, double* y, int64_t n, void* stream);

/* Fills *opts with the defaults listed at ba_options. */
ba_status ba_options_default(ba_options* opts);

/* Creates a problem from host index arrays (Sec. VI-A: cameras and points are the
 * tunable nodes, observations are constant and read sequentially).
 *   cam_idx[n_obs], pt_idx[n_obs]: host, camera / point of each observation.
 *   pixels[n_obs][2]: host, measured pixels.
 * Copied; the caller keeps ownership.  Requirements (else BA_ERR_INVALID_ARG):
 * 1 <= n_cams < 2^24, 1 <= n_pts, 1 <= n_obs < 2^32, every index in range, every
 * pixel finite, and every point observed at least twice.  No device memory is touched until
 * ba_bind_workspace. */
ba_status ba_problem_create(int32_t n_cams, int32_t n_pts, int64_t n_obs,
                            const uint32_t* cam_idx, const uint32_t* pt_idx,
                            const double* pixels, int32_t precision, ba_problem** out);

/* Frees the problem's host memory, streams and graphs (never the workspace). */
void ba_problem_destroy(ba_problem* problem);

/* Bytes of device workspace the problem needs (any options). */
ba_status ba_workspace_size(const ba_problem* problem, size_t* bytes);

/* Pose factors: generic node-to-node factors next to the reprojection factors
 * (Sec. IV of the paper: factors between nodes such as odometry / pose-graph
 * constraints).  Factor k ties cameras a = cam_a[k] and b = cam_b[k] (a != b) by a
 * measured relative pose: with world-to-camera maps x = R_c X + t_c,
 *   R_ba = R_b R_a^T,  t_ba = t_b - R_ba t_a,
 *   r_k = s_k * [ Log(Exp(w_m)^T R_ba) ; t_ba - t_m ]      (6 rows, elementwise s_k),
 * and the objective gains 1/2 sum_k |r_k|^2 (squared loss; a robust loss applies to
 * the observations only).  LM and PCG treat the factor rows like any other rows of J:
 * they enter g, the camera blocks of the preconditioner, D, the normal operator and
 * the model decrease.
 *   n_factors      >= 0; 0 removes every factor.
 *   cam_a, cam_b   host, [n_factors] camera indices < n_cams, cam_a[k] != cam_b[k].
 *   meas           host, [n_factors][6] FP64: w_m (rotation vector), t_m.
 *   sqrt_info      host, [n_factors][6] FP64 >= 0, the square root of a diagonal
 *                  information matrix; NULL = all ones.
 * The arrays are copied; the caller keeps ownership.  Call before ba_workspace_size
 * and ba_bind_workspace (the workspace holds the factors); a bound problem returns
 * BA_ERR_INVALID_ARG.  The mixed-precision form only (BA_ERR_NOT_IMPLEMENTED for
 * BA_PREC_FP64); ba_solve with solver = 1 (Schur complement) returns
 * BA_ERR_NOT_IMPLEMENTED when factors are present.  ba_evaluate's cost includes the
 * factors; its residual and Jacobian outputs, ba_cost_noalloc and the autograd entries
 * cover the observations only.  Invalid indices or non-finite values: INVALID_ARG. */
ba_status ba_set_pose_factors(ba_problem* problem, int32_t n_factors, const uint32_t* cam_a, const uint32_t* cam_b,
                              const double* meas, const double* sqrt_info);

/* Binds caller-owned device memory (>= ba_workspace_size bytes, 256-byte aligned)
 * and a CUDA stream (cudaStream_t, may be 0 for the legacy stream).  Uploads the
 * observations and builds the locality ordering on the device: points sorted by
 * their first camera, tiles of consecutive points, observations of a tile sorted
 * by camera (our counterpart of the Shared Read/Add index build of Sec. IV-A).
 * Must precede every call below.  Rebinding rebuilds everything. */
ba_status ba_bind_workspace(ba_problem* problem, void* workspace, size_t bytes, void* stream);

/* Parameters from / to host FP64 arrays in user layout. */
ba_status ba_set_params(ba_problem* problem, const double* cams, const double* pts);
ba_status ba_get_params(ba_problem* problem, double* cams, double* pts);

/* Parameters from / to device arrays in user layout; dtype 0 = float32, 1 = float64.
 * Enqueued on the bound stream, no synchronisation. */
ba_status ba_set_params_device(ba_problem* problem, const void* cams, const void* pts, int32_t dtype);
ba_status ba_get_params_device(ba_problem* problem, void* cams, void* pts, int32_t dtype);

/* Evaluates the problem at the current parameters (Sec. VI-A residual, Sec. V
 * Jacobian).  cost_out (host, may be NULL) receives 1/2 sum |r|^2 in FP64.
 * residuals (device, may be NULL): [n_obs][2] in the caller's observation order.
 * jacobian (device, may be NULL): [n_obs][2][12], columns = 9 camera parameters
 * then 3 point coordinates.  Element type float for BA_PREC_MIXED, double for
 * BA_PREC_FP64.  Synchronises when cost_out is given. */
ba_status ba_evaluate(ba_problem* problem, double* cost_out, void* residuals, void* jacobian);

/* Runs LM + PCGNR from the current parameters (Sec. V).  If stats is NULL the call
 * only enqueues the solve and returns; read results later with ba_get_stats.
 * Otherwise it synchronises and fills *stats and up to history_cap entries of
 * history (may be NULL). */
ba_status ba_solve(ba_problem* problem, const ba_options* opts, ba_stats* stats,
                   ba_iter_stat* history, int32_t history_cap);

/* Results of the last ba_solve (synchronises). */
ba_status ba_get_stats(ba_problem* problem, ba_stats* stats, ba_iter_stat* history,
                       int32_t history_cap);

/* Applies the damped normal operator once, out = (J^T J + mu D) v at the current
 * linearisation (Sec. V-A PCGNR step), for testing and kernel timing.  v and out are
 * device vectors in user layout (n_cams*9 then n_pts*3 entries, float for MIXED,
 * double for FP64).  Requires a prior ba_evaluate or ba_solve that linearised.
 * jp2_out (host, may be NULL) receives |J v|^2 + mu v^T D v in FP64 (synchronises). */
ba_status ba_apply_normal(ba_problem* problem, double mu, const void* v, void* out,
                          double* vAv_out);

/* Launches the normal-operator kernel `launches` times back to back on the bound
 * stream with the launch configuration the solver uses (timing aid). */
ba_status ba_repeat_normal(ba_problem* problem, int32_t launches);

/* Times each kernel of the solver in isolation with CUDA events on the bound stream:
 * `reps` launches each (after one warm-up launch), every launch timed alone with its
 * gates opened just before it, after a prior ba_evaluate or ba_solve.  Writes
 * the average microseconds per launch into us_out[0..n) in this order: camera
 * records, linearisation, preconditioner, normal operator (matvec), PCG update,
 * candidate step, candidate evaluation, commit; then [8] one launch of the persistent
 * PCG kernel (a whole PCG solve capped at 50 iterations with zero tolerance, each
 * launch after a preconditioner launch that resets its state, events around the PCG
 * launch alone) and [9] the PCG iterations that launch ran; -1 and 0 there when the
 * problem does not fit the persistent kernel; [10] one round of the one-reduction
 * separate-kernel PCG (pcg_kernel 3: camera update and direction records, pose
 * factors, tiles) past its first round, -1 when the tile kernels are not planned;
 * [11] the residual pass (all observations' residuals at the current parameters).
 * Leaves the solver state undefined
 * (the next ba_solve starts afresh).  Synchronises. */
ba_status ba_profile_kernels(ba_problem* problem, int32_t reps, double* us_out, int32_t n);

/* Total reprojection cost F = 1/2 sum |r|^2 (FP64 sum; residuals in the problem's
 * precision) at caller parameters, and its adjoint (Sec. V: the Jacobian of the
 * factor with respect to its tunable nodes).  cams/pts are device arrays in user
 * layout of dtype (0 float32, 1 float64).  Forward writes F to *cost_dev (device
 * double).  Backward recomputes the residuals and writes grad_cams = grad_out *
 * J_c^T r and grad_pts = grad_out * J_p^T r (device, same dtype, user layout), where
 * grad_out is a device double.  The problem's own parameters are not changed; the
 * backward reuses the linearisation buffers, so ba_apply_normal needs a new
 * ba_evaluate afterwards.  Neither call synchronises.  These back the
 * torch.autograd.Function of the Python binding. */
ba_status ba_cost_forward(ba_problem* problem, const void* cams, const void* pts, int32_t dtype,
                          double* cost_dev);
ba_status ba_cost_backward(ba_problem* problem, const void* cams, const void* pts, int32_t dtype,
                           const double* grad_out_dev, void* grad_cams, void* grad_pts);

/* Allocation-free cost, for callers that cannot allocate device memory: code that
 * runs while a stream is being captured into a CUDA graph, hosts whose device memory
 * belongs entirely to another allocator, or real-time loops in which allocation is
 * forbidden.  (The paper has no counterpart; this is a library service.)
 *
 * Computes F = 1/2 sum_o |r_o|^2 with the arithmetic of ba_evaluate for
 * BA_PREC_MIXED (FP32 residuals, FP64 sum) from caller-provided device arrays in user
 * layout: cams float[n_cams][9], pts float[n_pts][3], cam_idx / pt_idx uint32[n_obs],
 * pixels float[n_obs][2].  Indices are not validated on the host: every cam_idx must be
 * < n_cams and every pt_idx < n_pts; an observation whose index is out of range is
 * skipped without being read and makes the result NaN.  The result goes to *cost_dev
 * (device double).  Enqueued on
 * `stream` (cudaStream_t); no synchronisation, no cudaMalloc, no cudaFree and no
 * allocating library call.
 *
 * Scratch (camera records and per-block partial sums, about 1.1 MiB) is a fixed array
 * inside the library: every GPU that loads the library holds it until the process
 * exits.  Limits: n_cams <= BA_NOALLOC_MAX_CAMS and n_obs <= BA_NOALLOC_MAX_BLOCKS *
 * 1024; larger sizes are rejected with BA_ERR_INVALID_ARG before any GPU work.  Each
 * call made outside stream capture looks up the array's device address on the current
 * device (so a device reset is followed); a call under capture uses the address of the
 * last uncaptured call on that device, so make a first call on each device before any
 * stream capture (otherwise BA_ERR_STATE).  All calls share
 * the one array, so calls whose GPU work overlaps (other streams, other host threads
 * on the same device) race and must be serialised by the caller. */
#define BA_NOALLOC_MAX_CAMS 16384
#define BA_NOALLOC_MAX_BLOCKS 16384
ba_status ba_cost_noalloc(int32_t n_cams, int32_t n_pts, int64_t n_obs, const float* cams, const float* pts,
                          const uint32_t* cam_idx, const uint32_t* pt_idx, const float* pixels, double eps_depth,
                          double* cost_dev, void* stream);

/* ---- Batched mode ---------------------------------------------------------------
 * Many independent small problems (the uneven-size batch of the paper's evaluation,
 * Sec. VI) solved together by ONE persistent kernel: each CTA takes whole problems
 * from a device work queue, largest first, and runs the complete LM + PCGNR of Sec. V
 * for that problem with block-level synchronisation only.  Arithmetic as in
 * BA_PRECISION_MIXED (FP32 bulk, FP64 reductions and block inversions).  No CTA waits
 * on another, so the kernel has no inter-block spin-waits.
 *
 * ba_batch_create: host arrays, copied; the caller keeps ownership.
 *   cam_off, pt_off: int32 prefix offsets [n_problems + 1] into the concatenated
 *   camera and point arrays; obs_off: int64 prefix offsets into the observations.
 *   cam_idx / pt_idx [obs_off[n_problems]] are LOCAL to each problem (camera index <
 *   its camera count, point index < its point count); pixels [n_obs][2] FP64.
 *   Limits per problem: 1..BA_BATCH_MAX_CAMS cameras, 1..BA_BATCH_MAX_PTS points,
 *   every point observed at least twice; otherwise BA_ERR_INVALID_ARG.
 * ba_batch_workspace_size / ba_batch_bind_workspace: one device arena (256-byte
 *   aligned) and a borrowed stream, as for ba_problem.  Binding sorts the observations
 *   on the device by problem and camera (points in a per-camera rotated order) and builds the point-major index; it fails
 *   with BA_ERR_INVALID_ARG if the largest problem's shared-memory tables (376 bytes
 *   per camera + 12 bytes per point) do not fit one CTA.  Binding selects the default
 *   schedule (256 threads, occupancy-limited CTAs per SM).
 * ba_batch_set_params / ba_batch_get_params: host FP64, cameras [total_cams][9] and
 *   points [total_pts][3] in the concatenated order of ba_batch_create.  Synchronous.
 * ba_batch_solve: solves every problem with the same options (use_graph != 0: the
 *   work-queue reset and the persistent launch run as one captured CUDA graph, rebuilt
 *   when options or schedule change; pcg_kernel is ignored).  stats_per_problem NULL =
 *   asynchronous on the bound stream; otherwise an array of n_problems entries that is
 *   filled after a synchronisation (solve_ns = 0, no per-iteration history).
 * ba_batch_get_costs: initial and final cost of every problem of the last solve
 *   (either pointer may be NULL).  Synchronous.
 * ba_batch_set_schedule: threads per CTA (128, 256 or 512), resident CTAs per SM
 *   (0 = as many as occupancy allows; larger values are capped there) and flags:
 *   BA_SCHED_STAGE_POINTS keeps the points' parameters and search directions in
 *   shared memory during PCG (256 or 512 threads; needs 376 bytes per camera + 36 bytes
 *   per point of the largest problem per CTA, else BA_ERR_INVALID_ARG).
 * ba_batch_get_schedule: the current schedule and the resulting grid size.  Binding
 *   selects 512 threads with staged points when they fit, else 256 threads.
 * ba_batch_autotune: times one full solve per candidate schedule (every compiled block
 *   size at each CTAs-per-SM count its occupancy allows, with and without staged points)
 *   from the current parameters, restores the parameters,
 *   and keeps the fastest schedule.  Choices are cached for the life of the process,
 *   keyed by the GPU's name, the batch shape and the iteration options; a cached key
 *   applies its schedule without timing unless flags has BA_TUNE_IGNORE_CACHE.
 *   trials (capacity trial_cap, may be NULL when trial_cap = 0) receives the timings;
 *   *n_trials the number written (0 on a cache hit).  Synchronous. */
#define BA_BATCH_MAX_CAMS 1024
#define BA_BATCH_MAX_PTS 16384
#define BA_TUNE_IGNORE_CACHE 1
#define BA_SCHED_STAGE_POINTS 1
typedef struct ba_batch ba_batch;
typedef struct ba_batch_trial {
    int32_t threads, ctas_per_sm, flags, grid;
    float ms;
} ba_batch_trial;
ba_status ba_batch_create(int32_t n_problems, const int32_t* cam_off, const int32_t* pt_off,
                          const int64_t* obs_off, const uint32_t* cam_idx, const uint32_t* pt_idx,
                          const double* pixels, ba_batch** out);
void ba_batch_destroy(ba_batch* batch);
ba_status ba_batch_workspace_size(const ba_batch* batch, size_t* bytes);
ba_status ba_batch_bind_workspace(ba_batch* batch, void* workspace, size_t bytes, void* stream);
ba_status ba_batch_set_params(ba_batch* batch, const double* cams, const double* pts);
ba_status ba_batch_get_params(ba_batch* batch, double* cams, double* pts);
ba_status ba_batch_solve(ba_batch* batch, const ba_options* opts, ba_stats* stats_per_problem);
ba_status ba_batch_get_costs(ba_batch* batch, double* initial_costs, double* final_costs);
ba_status ba_batch_set_schedule(ba_batch* batch, int32_t threads, int32_t ctas_per_sm, int32_t flags);
ba_status ba_batch_get_schedule(const ba_batch* batch, int32_t* threads, int32_t* ctas_per_sm, int32_t* flags,
                                int32_t* grid);
ba_status ba_batch_autotune(ba_batch* batch, const ba_options* opts, int32_t flags, ba_batch_trial* trials,
                            int32_t trial_cap, int32_t* n_trials);

#ifdef __cplusplus
}
#endif
#endif /* GBBA_H */
