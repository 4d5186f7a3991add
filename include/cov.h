/*
 * cov.h -- C-ABI of the B300 (sm_103a) coverage-field library, libcov.so.
 *
 * Coverage trajectory synthesis as statistical inference (Sun, Kwon,
 * Murphey, arXiv 2511.11514).  A trajectory s_0..s_T is read as the sample
 * set {s_1..s_T} with weights a_i = 1/T (Eq. 1).  Each outer iteration
 *   1. evaluates a coverage flow field a_i = g(x_i) at all T samples at once
 *      (Sec. II-B, "Parallelized flow evaluation"), either the Stein
 *      variational field (Eq. 4) or the Sinkhorn-divergence field (Eq. 6-7);
 *   2. tracks the field with the LQR problem of Eq. 9-10 on the linearised
 *      dynamics of Eq. 8, giving a control direction v*;
 *   3. updates u <- u + eta v* and rolls the dynamics out again (Sec. II-C).
 *
 * Conventions shared by every call below:
 *   - Array arguments are caller-owned DEVICE pointers (e.g. the data_ptr()
 *     of a contiguous torch tensor on the context's device), row-major, with
 *     the shapes given in brackets.  Small descriptors (cov_gmm, Q, R,
 *     cov_problem) are host memory and are read during the call.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream).  Inputs must stay alive until the stream reaches the
 *     call.  Argument errors are returned synchronously and nothing is
 *     launched.  Device-detected conditions (non-finite values, a wait that
 *     ran out of its iteration limit, a non-SPD Riccati matrix) set bits in a
 *     device status word read by cov_get_device_status().
 *   - All device scratch memory is the context's workspace.  The workspace is
 *     allocated only by cov_ctx_create / cov_ctx_reserve*; no other call
 *     allocates.  A call whose sizes need more workspace than reserved
 *     returns COV_ERR_WORKSPACE without launching.
 *   - The library never aborts, prints or traps.  One context must not be
 *     used from two host threads at the same time, and two calls on the same
 *     context must not overlap on the GPU (they share the workspace): issue
 *     them on one stream, or synchronise between streams.
 *   - Precision: fields are computed in FP32 (exponentials through the
 *     ex2.approx special-function unit), the LQR step and the rollout in
 *     FP64.
 */
#ifndef COV_H
#define COV_H

#include <stddef.h>

#if defined(__GNUC__)
#define COV_API __attribute__((visibility("default")))
#else
#define COV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cov_stream_t; /* == cudaStream_t */
typedef struct cov_ctx cov_ctx;

typedef enum {
    COV_OK = 0,
    COV_ERR_INVALID_ARG = 1, /* bad size, pointer, or parameter value */
    COV_ERR_WORKSPACE = 2,   /* workspace too small / allocation failed */
    COV_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    COV_ERR_NONFINITE = 4,   /* device status: NaN/Inf or non-SPD matrix */
    COV_ERR_TIMEOUT = 5,     /* device status: a bounded wait gave up */
    COV_ERR_UNSUPPORTED = 6  /* size/dimension combination not built */
} cov_status;

/* Dynamics models: explicit Euler s_{t+1} = s_t + dt f(s_t, u_t).
 *   COV_SINGLE_INT  s = (p0, p1),          u = (u0, u1)           n=2, m=2
 *   COV_DOUBLE_INT  s = (p0, p1, v0, v1),  u = (acc0, acc1)       n=4, m=2
 *   COV_UNICYCLE    s = (x, y, theta),     u = (speed, turn rate) n=3, m=2 */
enum { COV_SINGLE_INT = 0, COV_DOUBLE_INT = 1, COV_UNICYCLE = 2 };
enum { COV_FIELD_SVGD = 0, COV_FIELD_SINKHORN = 1 };
/* cov_field_sinkhorn flags */
enum { COV_WARM_START = 1 };
/* device status bits (cov_get_device_status) */
enum { COV_DEV_NONFINITE = 1, COV_DEV_TIMEOUT = 2, COV_DEV_NOT_SPD = 4 };

#define COV_MAX_D 6        /* coverage dimensions of a field */
#define COV_MAX_GMM 32     /* mixture components */
#define COV_MAX_N 4        /* LQR state dimension */
#define COV_MAX_M 3        /* LQR control dimension */

/* Isotropic Gaussian mixture q(x) = sum_k w_k N(x; mu_k, sigma_k^2 I), the
 * reference of the Stein field (Sec. II-A: q given as a density).  Host
 * memory; the weights are normalised by the library. */
typedef struct {
    int K;              /* 1..COV_MAX_GMM */
    int d;              /* dimension, equal to the field's d */
    const float* w;     /* [K]   positive weights */
    const float* mu;    /* [K][d] means */
    const float* sigma; /* [K]   standard deviations, > 0 */
} cov_gmm;

/* ---- context and workspace --------------------------------------------- */

/* Create a context on `device` (the CUDA device ordinal).  Allocates the
 * device status word and `workspace_bytes` of workspace (0 = none yet). */
COV_API cov_status cov_ctx_create(cov_ctx** out, int device, size_t workspace_bytes);
/* Free the context and its workspace.  Safe on NULL.  Synchronises the
 * device first so no call still uses the workspace. */
COV_API void cov_ctx_destroy(cov_ctx* ctx);
/* Grow the workspace to at least `bytes` (never shrinks).  Synchronises the
 * device before freeing an old workspace. */
COV_API cov_status cov_ctx_reserve(cov_ctx* ctx, size_t bytes);
/* Workspace bytes that any single-problem call on these sizes needs:
 * T samples, M reference samples (0 if none), d coverage dims, and LQR
 * state/control dims n, m (0 if no LQR step). */
COV_API size_t cov_workspace_size(int T, int M, int d, int n, int m);
/* cov_ctx_reserve(ctx, cov_workspace_size(T, M, d, n, m)). */
COV_API cov_status cov_ctx_reserve_for(cov_ctx* ctx, int T, int M, int d, int n, int m);
/* Synchronise `stream`, return the OR of COV_DEV_* bits raised since the
 * last read in *flags, and clear them.  Returns COV_ERR_NONFINITE or
 * COV_ERR_TIMEOUT if the corresponding bits were set, else COV_OK. */
COV_API cov_status cov_get_device_status(cov_ctx* ctx, cov_stream_t stream, int* flags);
/* Human-readable name of a status code (static storage). */
COV_API const char* cov_status_string(cov_status s);
/* Text of the last CUDA runtime error seen by this context ("" if none). */
COV_API const char* cov_last_cuda_error(cov_ctx* ctx);

/* Tuning knobs of the all-pairs kernels (see cov_autotune in the binding).
 * key: COV_OPT_* ; value: as documented.  Returns COV_ERR_INVALID_ARG for an
 * unknown key or an out-of-range value. */
enum {
    COV_OPT_ROWS_PER_THREAD = 1, /* 2, 4 or 8 (default 4; 2 and 8 built for d = 2) */
    COV_OPT_THREADS = 2,         /* threads per CTA: 128 (the only value built) */
    COV_OPT_CTAS_PER_SM = 3,     /* cap on resident CTAs per SM planned for, 1..8 (default 8; the register budget may allow fewer) */
    COV_OPT_USE_GRAPH = 4,       /* cov_solve: capture one outer iteration in a CUDA graph (default 1) */
    COV_OPT_SPIN_LIMIT = 5,      /* bounded-wait iteration limit, >= 0 (default 1<<22) */
    COV_OPT_TENSOR_CORES = 6,    /* Exponents of the Sinkhorn updates with a fixed row offset (d <= 3):
                                    1: tcgen05 kind::tf32 MMAs on TF32-split operands; 0: FP32 FMAs on
                                    the CUDA cores; 2 (default): the tensor cores for field evaluations
                                    whose launches are all of at least 2^30 pair evaluations (where they
                                    are faster), the CUDA cores otherwise.  The tensor-core exponent error
                                    grows with the size of the exponent terms, (extent / sqrt(eps ln 2))^2 */
    COV_OPT_BATCH_SHARE = 7      /* cov_solve_batched: percent (1..100) of the GPU's resident CTA slots that
                                    each problem's all-pairs launches are planned for (its column splits),
                                    since the batch's problems run side by side (default 12) */
};
COV_API cov_status cov_ctx_set_option(cov_ctx* ctx, int key, long long value);

/* Tile-shape autotuner of the all-pairs kernels: times the Sinkhorn
 * iteration on these inputs (as cov_field_sinkhorn, uniform start) for each
 * candidate (rows per thread, resident-CTA cap) in {(2,8), (4,8), (8,8),
 * (4,6), (2,6), (8,4)} with CUDA events on `stream`, as (t(2 + n
 * iterations) - t(2)) / n (median of 3; n = 20 below 2^30 pair evaluations
 * per iteration, 4 above), and applies the fastest to the context.
 * The shape only concerns the CUDA-core kernel, so the sweep runs with
 * COV_OPT_TENSOR_CORES off and restores the context's setting after it.
 * Synchronises the stream.  best_R, best_ctas_per_sm: host outputs (may be
 * NULL); sweep: host [6][3] (R, cap, microseconds per iteration) or NULL.
 * Workspace as cov_field_sinkhorn. */
COV_API cov_status cov_autotune_sinkhorn(cov_ctx* ctx, const float* x, int T,
                                         const float* y, const float* b, int M,
                                         int d, float eps, int* best_R,
                                         int* best_ctas_per_sm, double* sweep,
                                         cov_stream_t stream);

/* ---- reference score ----------------------------------------------------- */

/* score[i] = grad log q(x_i) for the mixture q (Eq. 4 needs only the score,
 * Sec. II-B).  x, score: [T][d] FP32 device; gmm: host descriptor. */
COV_API cov_status cov_gmm_score(cov_ctx* ctx, const float* x, int T, int d,
                         const cov_gmm* gmm, float* score,
                         cov_stream_t stream);

/* Score of a reference given as a density on a pixel grid (Sec. II-A: q as
 * a continuous function), d = 2: q is the bilinear interpolant of
 * map[iy][ix] with pixel centres at ((ix + 1/2)/W, (iy + 1/2)/H) on [0,1]^2,
 * each coordinate clamped to the outermost centres (outside them that
 * component of the score is 0), and score = grad q / q.
 *   map [H][W] FP32 device, positive (row iy = second coordinate), H, W >= 2
 *   x [T][2] FP32 device;  score [T][2] FP32 device */
COV_API cov_status cov_density_score(cov_ctx* ctx, const float* map, int H, int W,
                                     const float* x, int T, float* score,
                                     cov_stream_t stream);

/* ---- Stein variational field, Eq. 4 ------------------------------------- */

/* a_out[i] = 1/T sum_j [ k(x_j, x_i) score_j + grad_{x_j} k(x_j, x_i) ],
 * k(x, x') = exp(-|x - x'|^2 / (2 h^2)) (the radial basis kernel of Sec.
 * II-B; the j = i term included).
 *   x      [T][d] FP32 device, 1 <= T, 1 <= d <= COV_MAX_D
 *   score  [T][d] FP32 device, or NULL: then gmm (host) gives the score
 *   h      kernel length-scale > 0
 *   a_out  [T][d] FP32 device */
COV_API cov_status cov_field_svgd(cov_ctx* ctx, const float* x, int T, int d,
                          const float* score, const cov_gmm* gmm, float h,
                          float* a_out, cov_stream_t stream);

/* Reverse mode of the Stein field for L = <abar, a> (Eq. 4; the product rule
 * over both roles of every point, row and column, of the all-pairs sum):
 *   sbar_l = dL/dscore_l = 1/T sum_j k_lj abar_j,
 *   xbar_l = 1/(T h^2) sum_j k_lj [ (abar_l - abar_j) - r_lj psi_lj ],
 *   r_lj = x_l - x_j, psi_lj = abar_l . s_j + abar_j . s_l + (abar_l - abar_j) . r_lj / h^2,
 * one all-pairs pass (one exponential and 6d + 3 FP32 operations per pair).
 *   x, abar [T][d] FP32 device;  h > 0
 *   score [T][d] FP32 device: then xbar is the gradient with the score held
 *          fixed and gmm, wbar, mubar, sigmabar are ignored; or NULL: the
 *          score is the mixture's (gmm, host descriptor, as cov_field_svgd)
 *          at x, xbar is the total gradient (kernel and score paths: the
 *          Hessian of log q applied to sbar is added), and the mixture
 *          gradients are written where the pointers are non-NULL:
 *          wbar [K] (raw weights; sum_k w_k wbar_k = 0), mubar [K][d],
 *          sigmabar [K], FP32 device (sums over the points in FP64)
 *   xbar [T][d] FP32 device, written;  sbar [T][d] FP32 device or NULL
 * Workspace: cov_workspace_size_svgd_vjp(T, d, K) (K = 0 with a given
 * score).  Errors: COV_ERR_INVALID_ARG for T < 1, d outside 1..COV_MAX_D,
 * h <= 0, NULL x/abar/xbar, or a NULL score without a valid mixture. */
COV_API size_t cov_workspace_size_svgd_vjp(int T, int d, int K);
COV_API cov_status cov_field_svgd_vjp(cov_ctx* ctx, const float* x, int T, int d,
                                      const float* score, const cov_gmm* gmm, float h,
                                      const float* abar, float* xbar, float* sbar,
                                      float* wbar, float* mubar, float* sigmabar,
                                      cov_stream_t stream);

/* ---- Sinkhorn-divergence field, Eq. 5-7 ---------------------------------- */

/* Log-domain Sinkhorn between p_s = (1/T) sum delta_{x_i} and
 * q = sum b_j delta_{y_j} with cost |x - y|^2 and entropic weight eps (the
 * paper's omega, Eq. 5), n_iter fixed iterations, each updating
 *   g_j = -eps LSE_i(log a_i + (f_i - c_ij)/eps)          (M rows over T)
 *   f_i = -eps LSE_j(log b_j + (g_j - c_ij)/eps)          (T rows over M)
 *   p_i = (p_i - eps LSE_k(log a_k + (p_k - c_ik)/eps))/2 (self term, Eq. 6)
 * then the debiased field (Eq. 7, descent direction scaled by 1/a_i)
 *   a_i = 2 (sum_j pi_ij y_j - sum_k pi^s_ik x_k),
 *   pi_ij  = softmax_j(log b_j + (g_j - c_ij)/eps),
 *   pi^s_ik = softmax_k(log a_k + (p_k - c_ik)/eps).
 *   x      [T][d] FP32 device;  y [M][d] FP32 device
 *   b      [M] FP32 device positive weights (normalised by the library),
 *          or NULL for uniform 1/M
 *   eps > 0, n_iter >= 0; flags: COV_WARM_START starts from the given
 *          f, g, p (all three non-NULL) instead of zeros
 *   f [T], g [M], p [T]  FP32 device potentials (cost units), written on
 *          return when non-NULL
 *   a_out  [T][d] FP32 device field, or NULL to skip the gradient pass
 * Errors: COV_ERR_INVALID_ARG for T<1, M<1, d outside 1..COV_MAX_D,
 * eps<=0, n_iter<0, NULL x/y, or warm start without f, g, p. */
COV_API cov_status cov_field_sinkhorn(cov_ctx* ctx, const float* x, int T,
                              const float* y, const float* b, int M, int d,
                              float eps, int n_iter, int flags, float* f,
                              float* g, float* p, float* a_out,
                              cov_stream_t stream);

/* Debiased Sinkhorn divergence of Eq. 6 after n_iter fixed iterations,
 * as its dual value, and its gradient with respect to the samples x:
 *   S = OT(p_s, q) - OT(p_s, p_s)/2 - OT(q, q)/2
 *     = <a, f> + <b, g> - <a, p> - <b, q_self>,
 * with f, g, p the potentials of cov_field_sinkhorn (cold start, n_iter
 * iterations) and q_self the reference's self potential after n_iter
 * averaged self updates over y; the sums run in FP64.  The gradient is the
 * envelope formula dS/dx_i = -(1/T) field_i (field of Eq. 7, exact at
 * convergence; at finite n_iter it is the gradient through the final
 * potentials held fixed).
 *   x [T][d], y [M][d] FP32 device;  b [M] FP32 device weights or NULL
 *   q_ref [M] FP32 device: with q_given = 1 the reference self potential
 *          of an earlier call on the same y, eps, n_iter (read, not
 *          recomputed: OT(q, q) does not depend on x); with q_given = 0 it
 *          is computed (an M x M self iteration) and written to q_ref, or
 *          kept in the workspace when q_ref is NULL
 *   value [1] FP64 device, written;  grad [T][d] FP32 device or NULL
 * Workspace: cov_workspace_size_divergence(T, M, d).  Errors as
 * cov_field_sinkhorn; COV_ERR_INVALID_ARG for q_given without q_ref or a
 * NULL value; COV_ERR_UNSUPPORTED for q_given = 0 with weights b (the self
 * potential of a weighted reference is not built: pass it in). */
COV_API size_t cov_workspace_size_divergence(int T, int M, int d);
COV_API cov_status cov_sinkhorn_divergence(cov_ctx* ctx, const float* x, int T,
                                           const float* y, const float* b, int M,
                                           int d, float eps, int n_iter, float* q_ref,
                                           int q_given, double* value, float* grad,
                                           cov_stream_t stream);

/* The same field with eps-scaling (annealing, a standard acceleration of
 * Sinkhorn at small eps; not in the paper): iteration t = 0..n_iter-1 runs
 * the three updates at eps_t = max(eps, eps_start eps_decay^t), carrying
 * the potentials over in cost units; the field and the returned potentials
 * are at eps.  eps_start <= eps is cov_field_sinkhorn.  Errors as
 * cov_field_sinkhorn, plus COV_ERR_INVALID_ARG for eps_decay outside (0, 1)
 * when eps_start > eps. */
COV_API cov_status cov_field_sinkhorn_annealed(cov_ctx* ctx, const float* x, int T,
                                               const float* y, const float* b, int M,
                                               int d, float eps, int n_iter,
                                               float eps_start, float eps_decay,
                                               int flags, float* f, float* g,
                                               float* p, float* a_out,
                                               cov_stream_t stream);

/* The same field for callers that must not allocate device memory.  The
 * paper has no counterpart: this is a library convenience.  Some programs
 * cannot call cudaMalloc: plugins whose host application owns every device
 * byte and hands it out from its own arena, or real-time loops that cannot
 * take the device-wide synchronisation that cudaMalloc/cudaFree imply.  This
 * entry point takes its scratch from one fixed 48 MiB array compiled into
 * the library (held on every GPU that loads it, until the process exits)
 * instead of a context workspace.  No context is needed and nothing is
 * allocated; the caller still passes x, y, b, f, g, p and a_out exactly as
 * for cov_field_sinkhorn, with the same meaning, and the results are those
 * of cov_field_sinkhorn with default options.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture begins.  Later calls use the cached address.
 *   - A call needs at most cov_workspace_size(T, M, d, 0, 0) bytes of the
 *     array; sizes whose scratch exceeds it are rejected with
 *     COV_ERR_WORKSPACE before anything is launched.  T = 65536 with
 *     M = 262144 fits at every d from 1 to COV_MAX_D (47.2 MiB at d = 6);
 *     at T = 65536 and d = 2, M up to 347136 fits.
 *   - Every call reuses the same array; the call clears what must start at
 *     zero on `stream` itself.  Calls that overlap on the GPU (different
 *     streams, or several host threads) race on the array: serialise them.
 *   - Device-detected conditions (non-finite values, a wait that gave up)
 *     are not reported; check the outputs for NaN/Inf instead. */
COV_API cov_status cov_field_sinkhorn_noalloc(const float* x, int T, const float* y,
                                              const float* b, int M, int d, float eps,
                                              int n_iter, int flags, float* f, float* g,
                                              float* p, float* a_out, cov_stream_t stream);

/* ---- dynamics (Eq. 3, 8) ------------------------------------------------ */

/* A_t = I + dt df/ds, B_t = dt df/du at (s_t, u_t), t = 0..T-1 (Eq. 8).
 *   s [T+1][n], u [T][m], A [T][n][n], B [T][n][m]: FP64 device. */
COV_API cov_status cov_linearize(cov_ctx* ctx, int model, const double* s,
                         const double* u, int T, double dt, double* A,
                         double* B, cov_stream_t stream);
/* s_0 = s0 (host [n]), s_{t+1} = s_t + dt f(s_t, u_t).
 *   u [T][m], s [T+1][n]: FP64 device.  For the linear models at T > 256
 *   the rollout runs chunked over the GPU and keeps its chunk totals in the
 *   context workspace when one is reserved (overwriting what cov_solve
 *   cached there, as the other workspace calls do). */
COV_API cov_status cov_rollout(cov_ctx* ctx, int model, const double* s0,
                       const double* u, int T, double dt, double* s,
                       cov_stream_t stream);

/* ---- LQR flow matching, Eq. 9-10 ---------------------------------------- */

/* Discrete-time LQR tracking of the reference flow (Eq. 9-10 on the time
 * grid; the common dt weight cancels):
 *   min_v sum_{t=1..T} |z_t - abar_t|_Q^2 + sum_{t=0..T-1} |v_t|_R^2,
 *   z_{t+1} = A_t z_t + B_t v_t, z_0 = 0,
 * by the backward Riccati recursion and a forward rollout, in FP64, both as
 * parallel-in-time scans over chunks of the horizon (horizons under 64 steps
 * run the serial Riccati recursion in one warp; short horizons of state
 * dimension 1 (T <= 1024) and 2 (T <= 512) run both affine recursions in
 * one thread block).
 *   A [T][n][n], B [T][n][m]  FP64 device
 *   Q [n][n] (PSD), R [m][m] (SPD)  FP64 HOST
 *   abar [T][n] FP64 device: row t-1 holds the target at time t = 1..T
 *   v_out [T][m] FP64 device;  z_out [T+1][n] FP64 device or NULL
 *   1 <= n <= COV_MAX_N, 1 <= m <= COV_MAX_M.  A Riccati matrix
 *   R + B'PB that is not positive definite raises COV_DEV_NOT_SPD. */
COV_API cov_status cov_lqr_track(cov_ctx* ctx, const double* A, const double* B,
                         const double* Q, const double* R, const double* abar,
                         int T, int n, int m, double* v_out, double* z_out,
                         cov_stream_t stream);

/* ---- outer iteration (Sec. II-C) ----------------------------------------- */

typedef struct {
    int model;            /* COV_SINGLE_INT / COV_DOUBLE_INT / COV_UNICYCLE */
    int T;                /* horizon: samples s_1..s_T */
    double dt;            /* Euler step */
    double s0[COV_MAX_N]; /* fixed initial state */
    int field;            /* COV_FIELD_SVGD or COV_FIELD_SINKHORN */
    int d;                /* coverage coordinates = first d state components */
    const float* y;       /* Sinkhorn: [M][d] FP32 device reference samples */
    const float* b;       /* Sinkhorn: [M] FP32 device weights or NULL */
    int M;
    float eps;            /* Sinkhorn entropic weight */
    int n_iter;           /* Sinkhorn iterations per field (cold start) */
    cov_gmm gmm;          /* SVGD reference (host descriptor) */
    float h;              /* SVGD kernel length-scale */
    double Q[COV_MAX_N * COV_MAX_N]; /* [n][n] tracking weight, row-major */
    double R[COV_MAX_M * COV_MAX_M]; /* [m][m] control weight, row-major */
    double eta;           /* control step size (u <- u + eta v*) */
    /* Sinkhorn variants (not in the paper; zero-initialise for the paper's
     * cold fixed-eps iterations): */
    float eps_start;      /* eps-scaling: iteration t runs at
                           * max(eps, eps_start eps_decay^t); <= eps: none */
    float eps_decay;      /* in (0, 1) when eps_start > eps */
    int warm;             /* 1: each field evaluation starts from the
                           * potentials of the previous outer iteration
                           * (cov_solve starts cold; cov_solve_continue keeps
                           * them while nothing else ran on the context) */
    /* Stein field with a pixel-density reference instead of gmm (d = 2):
     * [density_h][density_w] FP32 device map, as cov_density_score; NULL: gmm */
    const float* density;
    int density_h, density_w;
} cov_problem;

/* Run n_outer outer iterations: x = first d components of s_1..s_T;
 * field a; abar = a lifted to the state (zero on other components); A, B at
 * (s, u); v* = LQR(abar); u += eta v*; s = rollout(s0, u).
 *   u     [T][m]   FP64 device, in/out (the control)
 *   s_out [T+1][n] FP64 device, out (the trajectory after the last update)
 * With COV_OPT_USE_GRAPH (default) one outer iteration is captured in a
 * CUDA graph on first use and replayed; the graph is rebuilt when the
 * problem, pointers or sizes change. */
COV_API cov_status cov_solve(cov_ctx* ctx, const cov_problem* prob, int n_outer,
                     double* u, double* s_out, cov_stream_t stream);

/* Continue a solve: like cov_solve, but `s` must already hold the rollout of
 * `u` from s0 (as left by a previous cov_solve / cov_solve_continue call, or
 * restored from a checkpoint of (u, s)), so no initial rollout is done.
 *   u [T][m] FP64 device in/out;  s [T+1][n] FP64 device in/out. */
COV_API cov_status cov_solve_continue(cov_ctx* ctx, const cov_problem* prob, int n_outer,
                                      double* u, double* s, cov_stream_t stream);

/* Batched outer iterations of n_probs independent problems (each as in
 * cov_solve: its own model, horizon, field kind, reference, weights).  One
 * outer iteration of every problem is captured once into a single CUDA graph
 * (one independent branch per problem) and the graph is launched n_outer
 * times, so one launch advances all problems and the GPU interleaves their
 * kernels.  Problem p uses its own region of the workspace (reserve
 * cov_workspace_size_batched bytes).  Results equal those of cov_solve on
 * each problem alone.
 *   probs [n_probs] host;  u[p] [T_p][m_p], s_out[p] [T_p+1][n_p] FP64 device
 *   (u and s_out are host arrays of device pointers). */
COV_API cov_status cov_solve_batched(cov_ctx* ctx, const cov_problem* probs, int n_probs,
                                     int n_outer, double* const* u, double* const* s_out,
                                     cov_stream_t stream);
/* Workspace bytes cov_solve_batched needs for these problems (0 if one of
 * them is invalid). */
COV_API size_t cov_workspace_size_batched(const cov_problem* probs, int n_probs);

/* ---- adjoints: gradients through the outer iteration --------------------- */

/* Vector-Jacobian product of the Sinkhorn-divergence field (the map
 * (x, y, b) -> a of cov_field_sinkhorn, cold start, n_iter iterations) with
 * abar: the exact reverse mode of the unrolled log-domain iterations
 * (differentiability of the Sinkhorn iterations, Sec. II-B).  Every forward
 * softmax is rebuilt from a recorded forward run (the potentials of every
 * iteration are kept), so each reverse step is one all-pairs pass:
 *   xbar = d<abar, a>/dx,  ybar = d<abar, a>/dy,  bbar = d<abar, a>/db
 * with b the raw (unnormalised) weights.
 *   x [T][d], y [M][d], abar [T][d] FP32 device;  b [M] FP32 device or NULL
 *   xbar [T][d], ybar [M][d] FP32 device, written
 *   bbar [M] FP32 device, written (ignored when b is NULL)
 *   1 <= d <= 3 (COV_ERR_UNSUPPORTED above), n_iter >= 0.
 * Workspace: cov_workspace_size_vjp(T, M, d, n_iter) bytes (the record of
 * n_iter iterations: about 4 (2 + d)(n_iter + 2)(T + M) bytes plus the
 * forward's own scratch). */
COV_API size_t cov_workspace_size_vjp(int T, int M, int d, int n_iter);
COV_API cov_status cov_field_sinkhorn_vjp(cov_ctx* ctx, const float* x, int T,
                                          const float* y, const float* b, int M,
                                          int d, float eps, int n_iter,
                                          const float* abar, float* xbar,
                                          float* ybar, float* bbar,
                                          cov_stream_t stream);

/* Vector-Jacobian product of cov_lqr_track's v(abar) (Eq. 9-10; v is linear
 * in abar): abar_bar = Q G (G'QG + R)^-1 vbar with z = G v, computed as the
 * same LQR with a linear control cost -2 vbar'w and no state target
 * (Riccati gains, then the two affine scans).
 *   A [T][n][n], B [T][n][m], vbar [T][m] FP64 device; Q, R FP64 HOST
 *   abar_bar [T][n] FP64 device, written (row t-1 pairs with abar row t-1)
 * Workspace: cov_workspace_size_lqr_vjp(T, n, m). */
COV_API size_t cov_workspace_size_lqr_vjp(int T, int n, int m);
COV_API cov_status cov_lqr_vjp(cov_ctx* ctx, const double* A, const double* B,
                               const double* Q, const double* R,
                               const double* vbar, int T, int n, int m,
                               double* abar_bar, cov_stream_t stream);

/* Vector-Jacobian product of cov_rollout at the trajectory s (Eq. 3, 8):
 *   lambda_T = sbar_T, lambda_t = A_t' lambda_{t+1} + sbar_t,
 *   ubar_t = B_t' lambda_{t+1}, s0bar = lambda_0,
 * with A_t, B_t the linearisation at (s_t, u_t), as a chunked scan.
 *   s [T+1][n], u [T][m], sbar [T+1][n] FP64 device
 *   ubar [T][m], s0bar [n] FP64 device, written
 * Workspace: cov_workspace_size_lqr_vjp(T, n, m). */
COV_API cov_status cov_rollout_vjp(cov_ctx* ctx, int model, const double* s,
                                   const double* u, int T, double dt,
                                   const double* sbar, double* ubar,
                                   double* s0bar, cov_stream_t stream);

/* cov_solve that also keeps the checkpoints of a later cov_solve_backward:
 * s_hist[k] = the trajectory entering outer iteration k, k = 0..n_outer-1.
 *   s_hist [n_outer][T+1][n] FP64 device (NULL only when n_outer = 0).
 * flags: 0, or COV_CKPT_RECORD to also keep, inside the workspace, the
 *   record of every outer iteration's Sinkhorn iterations (the potentials
 *   of each iteration, about 4 (2 + d)(n_iter + 2)(T + M) bytes per outer
 *   iteration) so that cov_solve_backward need not recompute them (Sinkhorn
 *   field on a time-invariant model, d <= 3; reserve
 *   cov_workspace_size_backward(prob, n_outer, COV_BACKWARD_RECORDED)).
 *   The records stay valid until another call writes workspace scratch
 *   (any call on this context other than cov_solve_backward with the same
 *   problem, n_outer and s_hist). */
enum { COV_CKPT_RECORD = 1 };
COV_API cov_status cov_solve_checkpointed(cov_ctx* ctx, const cov_problem* prob,
                                          int n_outer, double* u, double* s_out,
                                          double* s_hist, int flags,
                                          cov_stream_t stream);

/* Gradient of a scalar loss L(s^K) through n_outer = K outer iterations of
 * cov_solve started from the control u0 (Sec. II-C), for a Sinkhorn field
 * on a time-invariant model (COV_SINGLE_INT, COV_DOUBLE_INT; d <= 3;
 * COV_ERR_UNSUPPORTED otherwise: the unicycle's A_t, B_t depend on the
 * trajectory and would need second derivatives of the dynamics).  Reverse
 * (cold fixed-eps iterations only: warm or eps_start > eps is
 * COV_ERR_UNSUPPORTED).  Reverse
 * sweep over k = K..1: rollout adjoint, LQR adjoint (cov_lqr_vjp), field
 * adjoint (cov_field_sinkhorn_vjp, recomputing the inner Sinkhorn
 * iterations from the checkpoint s^{k-1}).
 *   u0     [T][m] FP64 device: the control the forward started from
 *   s_hist [K][T+1][n] FP64 device checkpoints from cov_solve_checkpointed,
 *          or NULL: they are rebuilt by replaying the forward (K-1 extra
 *          outer iterations)
 *   sbar_K [T+1][n] FP64 device: dL/ds^K
 *   ybar [M][d] FP32 device, bbar [M] FP32 device (NULL allowed only when
 *          prob->b is NULL), written: dL/dy, dL/db
 *   s0bar [n] FP64 device, written: dL/ds_0;  u0bar [T][m] FP64 device or
 *          NULL, written: dL/du0
 * When the last call on the context was cov_solve_checkpointed with
 * COV_CKPT_RECORD on the same problem, n_outer and s_hist, the recorded
 * Sinkhorn iterations are used instead of recomputed (same results).
 * Workspace: cov_workspace_size_backward(prob, K, mode) with mode
 * COV_BACKWARD_CHECKPOINTS (s_hist given), COV_BACKWARD_REPLAY (s_hist NULL)
 * or COV_BACKWARD_RECORDED (after a recording forward). */
enum { COV_BACKWARD_CHECKPOINTS = 0, COV_BACKWARD_REPLAY = 1, COV_BACKWARD_RECORDED = 2 };
COV_API size_t cov_workspace_size_backward(const cov_problem* prob, int n_outer, int mode);
COV_API cov_status cov_solve_backward(cov_ctx* ctx, const cov_problem* prob,
                                      int n_outer, const double* u0,
                                      const double* s_hist, const double* sbar_K,
                                      float* ybar, float* bbar, double* s0bar,
                                      double* u0bar, cov_stream_t stream);

/* Gradient of a scalar loss L(s^K) through K = n_outer outer iterations of a
 * Stein-field solve (Eq. 4, Sec. II-C) with a Gaussian-mixture reference on
 * a time-invariant model (COV_SINGLE_INT, COV_DOUBLE_INT; a pixel-density
 * reference or the unicycle is COV_ERR_UNSUPPORTED): the reverse sweep of
 * cov_solve_backward with the Stein field's reverse mode (cov_field_svgd_vjp
 * through the mixture score) in place of the Sinkhorn one.
 *   u0, s_hist, sbar_K, s0bar, u0bar as cov_solve_backward (s_hist from
 *          cov_solve_checkpointed without COV_CKPT_RECORD, or NULL: rebuilt
 *          by replaying the forward)
 *   wbar [K], mubar [K][d], sigmabar [K] FP32 device or NULL, written: dL with
 *          respect to the mixture's raw weights, means and standard
 *          deviations (prob->gmm), summed over the outer iterations
 * Workspace: cov_workspace_size_backward(prob, K, COV_BACKWARD_CHECKPOINTS
 * or COV_BACKWARD_REPLAY). */
COV_API cov_status cov_solve_backward_svgd(cov_ctx* ctx, const cov_problem* prob,
                                           int n_outer, const double* u0,
                                           const double* s_hist, const double* sbar_K,
                                           float* wbar, float* mubar, float* sigmabar,
                                           double* s0bar, double* u0bar, cov_stream_t stream);

/* ---- measurement -------------------------------------------------------- */

/* Issue-rate probes for the roofline of the all-pairs kernels: each runs
 * `iters` dependent-chain iterations per thread on a full grid and reports
 * operations per second measured with CUDA events on `stream` (host
 * results, synchronises).  out[0] = FP32 FFMA lane-ops/s, out[1] = packed
 * f32x2 FMA lane-ops/s (two per instruction), out[2] = ex2.approx lane-ops/s,
 * out[3] = FP64 DFMA lane-ops/s, out[4] = FP64 DFMA dependent latency in
 * SM clock cycles, out[5] = SM clock (MHz) estimated over the probe,
 * out[6] = 2^x values/s computed on the FMA pipe (polynomial, no MUFU),
 * out[7] = that polynomial's largest relative error against FP64 exp2 on
 * [-125, 127].  out: 8 doubles. */
COV_API cov_status cov_probe_peaks(cov_ctx* ctx, int iters, double* out, cov_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* COV_H */
