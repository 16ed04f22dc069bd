/*
 * exact.h -- C ABI of the EXACT hot path on one GB300 (sm_103a).
 *
 * EXACT is the projected extragradient method (Eq. (11)) for the monotone
 * variational inequality with operator
 *     F(x) = (1/m) sum_{w,i} (y_{w,i} - I0 h_w(<a_i, x>)) a_i,      Eq. (8)
 *     h_w(t) = sum_k S[w][k] exp(-mu_k max(t, 0)),                    Eq. (7)
 * of single-material polychromatic CT (Sec. 1.2), with a Joseph ray-driven
 * projector standing in for the paper's Radon-derived rows a_i (Sec. 1,
 * notation list) and m = W * n the number of (window, ray) measurements.
 *
 * Conventions shared by every call:
 *  - Images are FP32 (FP64 inside exact_norm_estimate and on the dense
 *    exact_dense_* path), row-major
 *    [ny][nx]; pixel (ix, iy) has its centre at ((ix-(nx-1)/2) p, (iy-(ny-1)/2) p)
 *    with p = geometry.pixel.
 *  - Sinograms are [n_views][n_bins] (bins fastest); counts are
 *    [n_windows][n_views][n_bins], FP32 or BF16.
 *  - View v has angle th = angle0 + v * angle_range / n_views; the source-side
 *    unit vector is es = (cos th, sin th), the detector axis eu = (-sin th, cos th),
 *    bin b sits at u_b = (b - (n_bins-1)/2) * bin_pitch + det_offset along eu.
 *    Parallel beam: the ray passes through u_b * eu with direction -es.  Fan
 *    beam: the ray joins the source R_s * es to the flat-detector point
 *    (R_s - R_d) * es + u_b * eu  (R_s = src_to_center, R_d = src_to_det).
 *  - A[i][(j,k)] = delta_i * max(0, 1 - |t_i(j) - k|): j runs over pixel centre
 *    lines of the ray's driving axis (x when |dir_x| >= |dir_y|, else y),
 *    t_i(j) is the cross-axis pixel-index coordinate of the crossing and
 *    delta_i = p / |dir_drive|; pixels outside the image are zero.
 *  - All device pointers are caller-owned and stay caller-owned.  A plan owns
 *    only its ray/view tables (device memory it allocates at creation) and a
 *    small pinned host buffer; per-call scratch lives in a caller-allocated
 *    workspace bound with exact_plan_bind_workspace.
 *  - Calls taking a stream enqueue work on it and return without waiting,
 *    except those that hand a device result to the host (the norm
 *    estimates, the autotuners), which synchronise; so do the create and
 *    destroy calls.
 *    Every call validates its arguments and returns a status; none aborts,
 *    traps or prints.  A plan is used from one host thread at a time and on
 *    the device that was current when it was created.
 */
#ifndef EXACT_H
#define EXACT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
struct CUstream_st;
typedef struct CUstream_st *exact_stream_t;

typedef enum {
    EXACT_OK = 0,
    EXACT_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is out of range */
    EXACT_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed */
    EXACT_ERR_OOM = 3,         /* device or pinned memory could not be allocated */
    EXACT_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
    EXACT_ERR_NONFINITE = 5,   /* a NaN/Inf residual norm stopped a solve */
    EXACT_ERR_UNSUPPORTED = 6, /* valid input outside what the library supports */
    EXACT_ERR_NO_WORKSPACE = 7 /* the call needs a bound workspace */
} exact_status;

typedef enum { EXACT_F32 = 0, EXACT_BF16 = 1 } exact_dtype;

/* Scan geometry.  beam: 0 parallel, 1 fan (flat detector).  Lengths share one
 * unit (pixel, bin_pitch, det_offset, src_to_center, src_to_det); angles are
 * radians.  Requirements: 1 <= nx, ny <= 16384; n_views, n_bins >= 1;
 * n_views * n_bins <= 2^31 - 1; pixel, bin_pitch > 0; for a fan beam
 * src_to_det > src_to_center > half the image diagonal (the source stays
 * outside the image). */
typedef struct {
    int beam;
    int nx, ny;
    double pixel;
    int n_views;
    double angle0, angle_range;
    int n_bins;
    double bin_pitch, det_offset;
    double src_to_center, src_to_det;
} exact_geometry;

/* Energies: mu[k] > 0 is the attenuation per unit length at density 1 of
 * energy bin k (the paper's mu_j, Sec. 1.2), 1 <= n_energy <= EXACT_MAX_ENERGY. */
#define EXACT_MAX_ENERGY 256
typedef struct {
    int n_energy;
    const double *mu;
} exact_spectrum;

/* Detector windows: S[w * n_energy + k] >= 0 is the fraction of the source
 * intensity I0 that window w records from energy bin k, i.e. the paper's
 * (I_w / I0) s_{w,k} (Eq. (2), Sec. 1); each window needs some S > 0.
 * 1 <= n_windows <= 64. */
typedef struct {
    int n_windows;
    const double *S;
} exact_windows;

typedef struct exact_plan *exact_plan_t;

/* Build a plan: validate the parameters (Sec. 1.2: mu_k > 0, S >= 0), build
 * the per-ray Joseph tables and per-view back-projection tables in FP64 on
 * the host and upload them (FP32 and FP64 copies) to the current device.
 * Copies every host input; the caller may free them afterwards.
 * Synchronises.  *out is NULL on failure. */
exact_status exact_plan_create(const exact_geometry *geometry, const exact_spectrum *spectrum,
                               const exact_windows *windows, exact_plan_t *out);

/* Free the plan's tables and host buffers (not the workspace).  NULL is OK.
 * The caller must make sure no work using the plan is still in flight. */
exact_status exact_plan_destroy(exact_plan_t plan);

/* Number of rays n = n_views * n_bins and pixels d = nx * ny (either pointer
 * may be NULL). */
exact_status exact_plan_dims(exact_plan_t plan, long long *n_rays, long long *n_pixels);

/* Bytes of device workspace the plan needs (256-byte aligned start). */
size_t exact_plan_workspace_bytes(exact_plan_t plan);

/* Bind caller-owned device memory of at least exact_plan_workspace_bytes as
 * the plan's workspace (NULL, 0 unbinds).  The memory must stay valid while
 * calls using it are in flight; calls on one plan share it, so they must be
 * serialised on one stream (or synchronised). */
exact_status exact_plan_bind_workspace(exact_plan_t plan, void *dev_ptr, size_t bytes);

/* z = A x.  x: device [ny][nx] FP32; z: device [n_views][n_bins] FP32.
 * Needs the workspace. */
exact_status exact_forward(exact_plan_t plan, const float *x, float *z, exact_stream_t stream);

/* g = A^T r for the matrix of exact_forward, evaluated as a deterministic
 * pixel-driven gather (fixed order, no atomics).  Both calls evaluate the
 * same entries delta_i max(0, 1 - |t_i(j) - k|), but the FP32 route to the
 * crossing t_i(j) differs (exact_forward anchors it per ray and per group of
 * driving lines, this call steps it from a neighbouring ray), so the two are
 * transposes of each other up to ~1e-6 pixel in t and FP32 summation order.
 * r: device [n_views][n_bins] FP32; g: device [ny][nx] FP32.  No workspace. */
exact_status exact_adjoint(exact_plan_t plan, const float *r, float *g, exact_stream_t stream);

/* F(x) of Eq. (8) with m = n_windows * n_rays.  y: device counts
 * [n_windows][n_views][n_bins] of type y_dtype; I0 > 0 the source intensity;
 * F: device [ny][nx] FP32.  Needs the workspace. */
exact_status exact_operator(exact_plan_t plan, const float *x, const void *y, exact_dtype y_dtype,
                            double I0, float *F, exact_stream_t stream);

/* Options of the projection onto the TV ball intersected with a box (Sec. 3.1,
 * implementation of projections): Dykstra's algorithm between
 * X1 = {x : ||x||_TV <= tau} and X2 = [lo, hi]^d, P_X1 approximated by the
 * TV-regularised problem argmin_x ||x - z||^2 + lam ||x||_TV with lam found by
 * bisection.  ||x||_TV is the isotropic total variation with forward
 * differences (zero past the last row and column); the regularised problem is
 * solved by fgp_iters steps of the fast gradient projection method on its
 * dual, warm-started from the previous solve of the same projection. */
typedef struct {
    int fgp_iters;      /* dual steps per regularised solve (default 40) */
    int max_bisect;     /* regularised solves per projection onto X1 (default 40) */
    int max_dykstra;    /* Dykstra rounds (default 50) */
    int pad;
    double tol_tv;      /* accept lam once | ||x||_TV - tau | <= tol_tv (default 0.01, Sec. 3.1) */
    double tol_dykstra; /* stop Dykstra once ||z_{k+1} - z_k|| <= tol_dykstra (default 1e-4, Sec. 3.1) */
    double lam0;        /* first lam of the bisection (<= 0: 1) */
} exact_tv_opts;

typedef struct {
    int rounds;          /* Dykstra rounds run */
    int solves;          /* regularised solves run */
    double lam;          /* lam of the last regularised solve */
    exact_status status; /* EXACT_OK or EXACT_ERR_TIMEOUT */
} exact_tv_info;

exact_tv_opts exact_tv_opts_default(void);

/* Device workspace exact_tv_project needs for an nx x ny image (about 52 bytes
 * per pixel).  0 if no CUDA device is current. */
size_t exact_tv_workspace_bytes(int nx, int ny);

/* x = P_X(z) for X = {||x||_TV <= tau} ∩ [lo, hi]^d (Sec. 3.1; the paper uses
 * the nonnegative orthant lo = 0, hi = +inf and tau = ||x_star||_TV).  z, x:
 * device [ny][nx] FP32 (distinct buffers); tau >= 0; lo <= hi; workspace:
 * device memory of at least exact_tv_workspace_bytes(nx, ny), caller-owned;
 * opts NULL means the defaults; info may be NULL.  One cooperative launch on
 * `stream`; synchronises the stream and returns EXACT_ERR_TIMEOUT if a grid
 * barrier of the launch gave up waiting (x is then not valid). */
exact_status exact_tv_project(int nx, int ny, const float *z, double tau, double lo, double hi,
                              const exact_tv_opts *opts, float *x, void *workspace, size_t workspace_bytes,
                              exact_tv_info *info, exact_stream_t stream);

/* ---- Dense measurement vectors (Sec. 2.2, Gaussian model; Sec. 3.2, Fig. 6) ----
 * The operator of Eq. (8) with an explicit FP64 matrix A whose rows are the
 * measurement vectors a_i (i.i.d. N(0, I_d) in the Gaussian model):
 *   F(x) = (1/(W n)) sum_{w,i} (y_{w,i} - I0 h_w(<a_i, x>)) a_i,
 * h_w as in Eq. (7) (the ReLU of Eq. (4) matters here: <a_i, x> can be
 * negative).  All arithmetic is FP64 (Fig. 6 follows the error to machine
 * precision); every sum has a fixed order. */
typedef struct exact_dense *exact_dense_t;

/* A: caller-owned device [n][d] FP64, row-major, kept by pointer (it must
 * outlive the context and not change while work using it is in flight);
 * spectrum and windows as in exact_plan_create (copied).  The context
 * allocates its own scratch (8 (W K + K + n + d + ceil(n/64) d) bytes). */
exact_status exact_dense_create(int n, int d, const double *A, const exact_spectrum *spectrum,
                                const exact_windows *windows, exact_dense_t *out);
exact_status exact_dense_destroy(exact_dense_t dense);

/* F(x): x device [d], y device [W][n], F device [d], all FP64. */
exact_status exact_dense_operator(exact_dense_t dense, const double *x, const double *y, double I0, double *F,
                                  exact_stream_t stream);

/* `iters` iterations of Eq. (11) on the box [lo, hi]^d (lo = -inf, hi = +inf:
 * no projection, as in Sec. 3.2) in place on x (device [d]).  If x_true
 * (device [d]) is given, err (device [iters]) receives ||x_t - x_true|| after
 * iteration t (both NULL otherwise).  Asynchronous on stream. */
exact_status exact_dense_solve(exact_dense_t dense, const double *y, double I0, double eta, int iters, double lo,
                               double hi, double *x, const double *x_true, double *err, exact_stream_t stream);

/* Kernel tuning of a plan (no counterpart in the paper: a property of this
 * implementation).  adj_split: CTAs sharing one 32 x 32-pixel tile of the
 * adjoint, each taking an interleaved subset of the views (1..16, and at most
 * the plan's limit: about 64 CTAs per SM in all, else EXACT_ERR_UNSUPPORTED;
 * the workspace holds one partial tile per split); the tile's partial sums
 * are added in split order, so results are deterministic for a given value
 * and differ only in FP32 rounding between values.  A new plan starts with
 * the largest of {1, 2, 3, 4, 6, 8, 12, 16} that keeps about 14 CTAs per SM.
 * reserved must be zero. */
typedef struct {
    int adj_split;
    int reserved[7];
} exact_tuning;

exact_status exact_plan_get_tuning(exact_plan_t plan, exact_tuning *out);
exact_status exact_plan_set_tuning(exact_plan_t plan, const exact_tuning *tuning);

/* Autotuner: times the adjoint of this plan's geometry on the device for
 * adj_split in {1, 2, 3, 4, 6, 8, 12, 16} within the plan's limit (9 rounds after a warm-up round, one launch
 * of each value per round; median per value) and keeps the fastest, a larger
 * split only when it is more than 1% faster.  The choice is
 * cached per geometry shape (beam, nx, ny, n_views, n_bins) for the life of
 * the process: later plans of a tuned shape take it without timing unless
 * force != 0.  out may be NULL.  Uses the plan's workspace as scratch;
 * synchronises the stream. */
exact_status exact_plan_autotune(exact_plan_t plan, int force, exact_tuning *out, exact_stream_t stream);

/* argmin_x ||x - z||^2 + lam ||x||_TV (the TV-regularised problem of Sec. 3.1,
 * and the step of the proximal variant of Sec. 5), by fgp_iters steps of the
 * fast gradient projection method from a zero dual.  z, x: device [ny][nx]
 * FP32, distinct; lam > 0; workspace as for exact_tv_project.  Synchronises. */
exact_status exact_tv_prox(int nx, int ny, const float *z, double lam, int fgp_iters, float *x, void *workspace,
                           size_t workspace_bytes, exact_stream_t stream);

/* Stopping rules of exact_solve (see exact_solve_opts). */
typedef enum {
    EXACT_STOP_RESIDUAL = 0, /* relative change of the iterate */
    EXACT_STOP_AVERAGE = 1   /* change of the running average of Sec. 3.1 */
} exact_stop_rule;

/* Options of exact_solve.  lo <= hi bound the box feasible set X = [lo, hi]^d
 * (lo = 0, hi = +inf is the nonnegative orthant of Sec. 3.1; lo = -inf
 * disables the lower bound); tv_bound > 0 intersects it with the TV ball of
 * Sec. 3.1 (each half and full step then projects with exact_tv_project's
 * algorithm, the bisection of each of the two projections starting from its
 * lam of the previous iteration; average_tail must be 0, else
 * EXACT_ERR_UNSUPPORTED).  prox_lambda > 0 selects the proximal variant the
 * Discussion (Sec. 5) proposes instead of the projection:
 *   x_{t+1/2} = argmin_x ||x - (x_t - eta F(x_t))||^2 + prox_lambda ||x||_TV,
 *   x_{t+1}   = argmin_x ||x - (x_t - eta F(x_{t+1/2}))||^2 + prox_lambda ||x||_TV,
 * each solved by tv.fgp_iters dual steps from a zero dual (exact_tv_prox);
 * there is no constraint then (lo, hi only clamp x_1; tv_bound must be 0).
 * Iterations are counted
 * t = 1, 2, ...; x_t is the iterate after t of them.
 *  - stop_rule EXACT_STOP_RESIDUAL: if tol > 0 and check_every > 0 the solve
 *    stops after the first t that is a multiple of check_every with
 *    rel_res = ||x_t - x_{t-1}|| / max(||x_{t-1}||, 1e-30) <= tol (FP64
 *    norms).  average_tail != 0 returns the mean of x_t for
 *    t > floor(iters/2) instead of the last iterate.
 *  - stop_rule EXACT_STOP_AVERAGE (Sec. 3.1, comparison of methods): the
 *    estimate at t is the mean xbar_t of the last m_t = max(1, floor(t/2))
 *    iterates x_{t-m_t+1} .. x_t; if tol > 0 and check_every > 0 the solve
 *    stops after the first t >= 2 that is a multiple of check_every with
 *    avg_change = ||xbar_t - xbar_{t-1}|| <= tol (absolute, FP64; the paper
 *    uses 1e-5), and returns xbar_T for the last iteration T run.  The running
 *    sum is kept in FP64, so xbar_t is the exact mean of the FP32 iterates up
 *    to one final rounding.  history: caller-owned device ring of history_cap
 *    images [ny][nx] FP32 holding the iterates of the window; history_cap >=
 *    max(1, floor(iters/2)).  average_tail must be 0. */
typedef struct {
    double lo, hi, tol;
    int check_every;
    int average_tail;
    int stop_rule;   /* exact_stop_rule */
    int history_cap; /* EXACT_STOP_AVERAGE: images in history */
    float *history;  /* EXACT_STOP_AVERAGE: device ring [history_cap][ny][nx] */
    double tv_bound; /* > 0: X = {||x||_TV <= tv_bound} ∩ [lo, hi]^d (see exact_tv_project) */
    exact_tv_opts tv; /* options of that projection */
    double prox_lambda; /* > 0: the proximal variant of the Discussion (see below) */
    /* Checkpoint / resume (no counterpart in the paper: the iteration of
     * Eq. (11) only needs x_t, plus the averaging sums and the TV bisection's
     * lam pair when those are in use).  The call runs iterations
     * t0 + 1 .. t0 + iters; with t0 > 0, x holds the last iterate of the call
     * that ran up to t0 (its x_last), and the averaging sums and lam pair are
     * continued from `resume` instead of being started afresh, so the iterates,
     * averages, stopping tests and info.iters_done (a total) are bitwise those
     * of one call of t0 + iters iterations, provided nothing else used that
     * state in between. */
    int t0;          /* iterations run by earlier calls of this solve (0: a fresh solve) */
    int total_iters; /* iterations of the whole solve, for average_tail's window (0: t0 + iters) */
    void *resume;    /* device, exact_solve_resume_bytes(plan) bytes, 8-byte aligned, caller-owned:
                      * the averaging sums and lam pair; NULL: kept in the workspace */
    float *x_last;   /* device [ny][nx] or NULL: receives the last iterate (x receives the average
                      * when an averaging option is on) */
    int launch;      /* 0: one CUDA graph whose WHILE node loops over the iterations on the device
                      * (the stopping test ends the loop; no launch runs after a stop) whenever the
                      * stream is not capturing, profiling is off and there is no TV ball or
                      * proximal step, else one stream launch per kernel; 1: always the latter */
    int pad;
} exact_solve_opts;

/* Bytes of the caller-owned resume state of exact_solve_opts.resume:
 * 8 (nx ny + 2). */
size_t exact_solve_resume_bytes(exact_plan_t plan);

typedef struct {
    int iters_done;      /* iterations run */
    double rel_res;      /* rel_res of the last iteration run (0 if none) */
    exact_status status; /* EXACT_OK or EXACT_ERR_NONFINITE */
    double avg_change;   /* EXACT_STOP_AVERAGE: ||xbar_T - xbar_{T-1}|| of the last
                          * iteration T run (0 if T < 2); else 0 */
} exact_solve_info;

/* Default options: lo = 0, hi = +inf, tol = 0, check_every = 1, average_tail = 0,
 * stop_rule = EXACT_STOP_RESIDUAL, no history, tv_bound = 0 (no TV ball),
 * tv = exact_tv_opts_default(), prox_lambda = 0, t0 = 0, total_iters = 0,
 * resume = NULL, x_last = NULL, launch = 0. */
exact_solve_opts exact_solve_opts_default(void);

/* Projected extragradient, Eq. (11), with constant step eta:
 *   x_{t+1/2} = P_X(x_t - eta F(x_t)),  x_{t+1} = P_X(x_t - eta F(x_{t+1/2})).
 * y: device counts as in exact_operator; x: device [ny][nx] FP32 holding x_1
 * on entry (projected onto X first) and the result on return; info: host
 * struct written once the stream reaches the end of the solve (valid after
 * synchronising the stream), may be NULL; opts NULL means the defaults.
 * Needs the workspace.  With opts.launch = 0 the plan keeps up to four
 * instantiated CUDA graphs, keyed by the kernel arguments that do not change
 * between calls of one reconstruction (I0, eta, bounds, averaging buffers,
 * split), so repeated calls (rounds of a server, resumed solves) relaunch one
 * graph; a new key may wait for the oldest graph's last launch to finish. */
exact_status exact_solve(exact_plan_t plan, const void *y, exact_dtype y_dtype, double I0, double eta,
                         int iters, const exact_solve_opts *opts, float *x, exact_solve_info *info,
                         exact_stream_t stream);

/* exact_solve from host memory: copies the counts y_host ([n_windows][n_views]
 * [n_bins] of type y_dtype) and x_1 from x_host ([ny][nx] FP32) into the
 * plan's workspace, runs exact_solve there and copies the result back into
 * x_host, all on `stream`, then synchronises it (so info is valid on return).
 * Host buffers may be pageable or pinned (pinned copies run at full bus
 * speed).  Not allowed while `stream` is being captured
 * (EXACT_ERR_UNSUPPORTED).  Needs the workspace. */
exact_status exact_solve_host(exact_plan_t plan, const void *y_host, exact_dtype y_dtype, double I0, double eta,
                              int iters, const exact_solve_opts *opts, float *x_host, exact_solve_info *info,
                              exact_stream_t stream);

/* ||A||_op^2 = lambda_max(A^T A) by FP64 power iteration on the device
 * (Sec. 4.2 needs lambda_max(Sigma) = ||A||^2 / n for the step size of
 * Theorem 2): v_1 = 1/sqrt(d), lam_k = ||A v_k||^2,
 * v_{k+1} = A^T A v_k / ||A^T A v_k||, stopping when
 * |lam_k - lam_{k-1}| <= rtol * lam_k or after max_iters (rtol = 0: exactly
 * max_iters iterations).  Synchronises.
 * iters_done may be NULL.  Needs the workspace. */
exact_status exact_norm_estimate(exact_plan_t plan, int max_iters, double rtol, double *normA_sq,
                                 int *iters_done, exact_stream_t stream);

/* The same power iteration with the FP32 projector kernels (FP64 norms and
 * Rayleigh quotients): ~1e-6 relative agreement with exact_norm_estimate at a
 * small fraction of its cost (FP64 arithmetic runs at a low rate on GB300);
 * used where a step size is needed per request.  Synchronises.  Needs the
 * workspace. */
exact_status exact_norm_estimate_f32(exact_plan_t plan, int max_iters, double rtol, double *normA_sq,
                                     int *iters_done, exact_stream_t stream);

/* Step size 1/(4L) of Theorem 1 with L = I0 (normA_sq / m) sum_k mu_k sum_w S[w][k]
 * (the Lipschitz bound of Sec. 4.2, m = n_windows * n_rays).  Host arithmetic. */
exact_status exact_recommended_eta(exact_plan_t plan, double I0, double normA_sq, double *eta);

/* F(x) as exact_operator computes it, for callers that cannot
 * allocate device memory when they need it: allocator-free real-time loops
 * that must not stall on cudaMalloc, and processes whose device memory is
 * owned by another framework's pool and cannot spare a separate workspace.  The paper has no counterpart: this is a
 * deployment variant of exact_operator.  Instead of the plan's bound workspace
 * it uses one file-scope device array of EXACT_STATIC_SCRATCH_MB MiB as
 * scratch, so the call allocates nothing and needs no workspace (the plan
 * itself, with its tables, is created beforehand).  The array exists once per
 * device that loads the library and lives until the process exits.
 *  - A plan whose scratch (padded image copies, collapsed counts, residual:
 *    about 8 (nx + 8)(ny + 8) + 8 n_views n_bins bytes) exceeds the array is
 *    rejected with EXACT_ERR_UNSUPPORTED.
 *  - The first call on a device looks the array's device address up (with that
 *    device current) and keeps it; make that first call before any stream
 *    capture.  cudaDeviceReset invalidates the kept address: do not call this
 *    entry point again in a process that reset the device.
 *  - The adjoint runs one CTA per 32 x 32 tile whatever the plan's
 *    exact_tuning.adj_split (a split needs the workspace), so F equals
 *    exact_operator's up to the FP32 summation order when adj_split > 1.
 *  - Every call shares the array and it keeps the last call's contents (each
 *    call writes all scratch it reads, so nothing has to be cleared); calls
 *    that overlap on the GPU -- other streams, other threads -- race on it.
 * Arguments, layouts and the other errors as exact_operator. */
#define EXACT_STATIC_SCRATCH_MB 24
exact_status exact_operator_static(exact_plan_t plan, const float *x, const void *y, exact_dtype y_dtype,
                                   double I0, float *F, exact_stream_t stream);

/* Known background (Appendix A.1: recover one material while the others are
 * known).  The rays also cross n_materials (0..4) known materials with
 * projections p, a device array [n_materials][n_views][n_bins] FP32 (e.g.
 * exact_forward of each known density), attenuating energy k by
 * exp(-mu_bg[m][k] p_m) with mu_bg[m * n_energy + k] >= 0 (host, copied).  The
 * plan keeps the pointer p (caller-owned; it must stay valid and unchanged
 * while later operator/solve/batch calls on the plan run).  n_materials = 0
 * removes the background.  F stays monotone and the Lipschitz bound of
 * exact_recommended_eta still holds (the background only lowers each h_w). */
exact_status exact_plan_set_background(exact_plan_t plan, int n_materials, const double *mu_bg, const float *p);

/* ---- Batched solves (many reconstructions in one persistent launch) ---- */

typedef struct exact_batch *exact_batch_t;

/* One reconstruction of a batch: a plan with its bound workspace (each job
 * needs its own plan and workspace), device counts y as in exact_operator, the
 * source intensity, the step, the iteration count, the options (average_tail
 * must be 0 and stop_rule EXACT_STOP_RESIDUAL, else EXACT_ERR_UNSUPPORTED), the
 * device image x (x_1 in, result out) and an optional host
 * info struct written when the stream reaches the end of the batch. */
typedef struct {
    exact_plan_t plan;
    const void *y;
    exact_dtype y_dtype;
    double I0;
    double eta;
    int iters;
    exact_solve_opts opts;
    float *x;
    exact_solve_info *info;
} exact_job;

/* Create a batch context for up to max_jobs (1..256) jobs per call: it owns a
 * few small device buffers (job descriptors, tensor maps, link coefficients,
 * work counters) and pinned host staging.  Synchronises. */
exact_status exact_batch_create(int max_jobs, exact_batch_t *out);

/* Free a batch context (no work using it may be in flight). */
exact_status exact_batch_destroy(exact_batch_t batch);

/* Run the projected extragradient iteration (Eq. (11)) of every job.  Under
 * the context's policy 0 or 1 (exact_batch_autotune, exact_batch_set_policy)
 * all jobs run in one persistent kernel launch: the work of all jobs (forward
 * units, adjoint tiles, reductions of each iteration) is handed out in a fixed
 * order through a device work counter; an item waits (bounded spin, then
 * EXACT_ERR_TIMEOUT) only for the previous phase of its own job, so different
 * jobs overlap.  Under policy 2 each job runs as its own exact_solve (graph
 * loop, the plan's adj_split) on one of the context's 8 streams, round robin,
 * forked from and joined back into `stream` with events, so jobs overlap
 * through the streams.  Per job the arithmetic is the same for any batch
 * composition, so a job's result does not depend on the other jobs (under
 * policy 2 it equals exact_solve's bit for bit).  Jobs on one call must be
 * distinct plans on the current device.  Asynchronous on `stream`;
 * capturable in a CUDA graph.  The context's staging is reused by the next
 * call, which waits for this call's staging copy first. */
exact_status exact_batch_solve(exact_batch_t batch, const exact_job *jobs, int n_jobs, exact_stream_t stream);

/* Autotuner of a batch context (no counterpart in the paper): times
 * exact_batch_solve on these jobs, two iterations each (best of two after a
 * warm-up run), under each policy -- 0: persistent kernel, one CTA per
 * adjoint tile; 1: persistent kernel, each plan's own exact_tuning.adj_split;
 * 2: one exact_solve per job on the context's streams -- and keeps the
 * fastest (a later policy only when more than 3% faster) for later
 * exact_batch_solve calls of this context.  Every job's x is saved in its plan's workspace and
 * restored after each trial, and the jobs' info structs are not written.
 * policy_out may be NULL.  Synchronises. */
exact_status exact_batch_autotune(exact_batch_t batch, const exact_job *jobs, int n_jobs, int *policy_out,
                                  exact_stream_t stream);

/* Set or read a batch context's policy (0, 1 or 2, as exact_batch_autotune;
 * a new context starts at 0).  No counterpart in the paper.  Set returns
 * EXACT_ERR_INVALID_ARG for another value. */
exact_status exact_batch_set_policy(exact_batch_t batch, int policy);
exact_status exact_batch_get_policy(exact_batch_t batch, int *policy);

/* Number of nonzero entries of A (pairs of ray and pixel with a positive
 * Joseph weight), counted in FP64 on the host at plan creation: the
 * algorithmic work of one forward or adjoint (one multiply-add per entry). */
exact_status exact_plan_nnz(exact_plan_t plan, long long *nnz);

/* Kernel timing of exact_solve, a profiling aid.  With sample_every > 0, every
 * sample_every-th iteration (t % sample_every == 0) of the following solves on
 * this plan records CUDA events around each of its kernels; 0 turns it off.
 * Returns EXACT_ERR_OOM if the plan's event pool cannot be created. */
#define EXACT_PROF_KINDS 4 /* 0 forward+link, 1 adjoint half step, 2 adjoint full step, 3 reduction */
exact_status exact_profile_enable(exact_plan_t plan, int sample_every);

/* Sum of the recorded kernel durations (ms) and number of timed launches per
 * kind since the last read; synchronises on the recorded events, then clears
 * them.  Either array may be NULL. */
exact_status exact_profile_read(exact_plan_t plan, double ms[EXACT_PROF_KINDS],
                                long long launches[EXACT_PROF_KINDS]);

/* Measurement aid (no counterpart in the paper): the rate, in 4-byte words per
 * second, at which the current device serves bank-conflict-free shared-memory
 * loads, measured by a kernel that issues only such loads on every SM (one full
 * wave, best of five launches timed with CUDA events on `stream`).  The
 * projector kernels gather one such operand per nonzero of A, so nonzeros per
 * second over this rate is their fraction of the on-chip gather ceiling.
 * sm_count (may be NULL) receives the device's SM count.  Synchronises. */
exact_status exact_probe_gather_ceiling(double *words_per_s, int *sm_count, exact_stream_t stream);

/* Fault injection for tests of the bounded device waits (no counterpart in the
 * paper).  Every device-side wait of this library -- the forward's staging
 * copies, the persistent batch kernel's waits for the previous phase of a job,
 * the TV projection's grid barriers -- gives up after a bounded number of polls
 * and reports EXACT_ERR_TIMEOUT instead of hanging; every thread block then
 * leaves and the device stays usable.  These switches let a test make such a
 * wait run out on purpose:
 *  - EXACT_INJECT_WAIT_POLLS, value >= 0: polls before a batch dependency wait
 *    or a TV grid barrier gives up (0: the built-in limits, seconds each);
 *  - EXACT_INJECT_BLOCK_BATCH_JOB, value = job index (-1: none): in the next
 *    exact_batch_solve that job's later phases wait for more completions than
 *    the job has items, so its wait runs out (EXACT_ERR_TIMEOUT in its info)
 *    and the launch ends;
 *  - EXACT_INJECT_BLOCK_TV_BARRIER, value != 0: the next TV projection launch
 *    (exact_tv_project, exact_tv_prox, or a solve with tv_bound / prox_lambda)
 *    starts its grid barrier's arrival count at the grid size, so the barrier
 *    never completes and the call reports EXACT_ERR_TIMEOUT.
 * The blocks are one-shot; the settings are process-wide. */
#define EXACT_INJECT_WAIT_POLLS 1
#define EXACT_INJECT_BLOCK_BATCH_JOB 2
#define EXACT_INJECT_BLOCK_TV_BARRIER 3
exact_status exact_debug_inject(int kind, long long value);

/* Static description of a status code. */
const char *exact_status_string(exact_status status);

#ifdef __cplusplus
}
#endif

#endif /* EXACT_H */
