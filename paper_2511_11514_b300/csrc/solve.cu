// solve.cu -- the outer iteration of Sec. II-C (cov_solve): coverage field on
// all samples, lift to the state space, linearise, LQR tracking, control
// update and rollout, repeated n_outer times on one stream.  One outer
// iteration is captured in a CUDA graph and replayed.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace cov {

int model_dims(int model, int* n, int* m);
size_t lqr_gain_doubles(int T, int n, int m);
cov_status lqr_riccati(cov_ctx* ctx, int n, int m, const double* A, const double* B, const double* Q,
                       const double* R, int T, double* gains, cudaStream_t stream);
cov_status lqr_step_single_int(cov_ctx* ctx, const double* B, const double* gains, const double* Q, const float* a,
                               int d, int T, double* v, double eta, double dt, const double* s0, double* u, double* s,
                               cudaStream_t stream);
cov_status lqr_affine(cov_ctx* ctx, void* ws, size_t ws_bytes, int n, int m, const double* B, const double* gains,
                      const double* Q, const double* abar, int T, double* v_out, double* z_out, cudaStream_t stream);
cov_status update_rollout(cov_ctx* ctx, int model, const double* s0, double* u, const double* v, double eta, int T,
                          double dt, double* s, cudaStream_t stream, double* scratch = nullptr);
size_t rollout_scratch_doubles(int T);
cov_status linearize_launch(cov_ctx* ctx, int model, const double* s, const double* u, int T, double dt, double* A,
                            double* B, cudaStream_t stream);

// Reference samples of a Sinkhorn problem (0 for the Stein field).
static int prob_M(const cov_problem* P) { return P->field == COV_FIELD_SINKHORN ? P->M : 0; }

// Time-invariant models: A_t, B_t do not depend on the trajectory, so the
// Riccati gains are the same in every outer iteration.
static bool model_is_lti(int model) { return model == COV_SINGLE_INT || model == COV_DOUBLE_INT; }

struct SolveBufs {
    float *x, *a, *scal;
    float *f, *g, *p;  // Sinkhorn potentials carried between outer iterations (warm)
    double *abar, *A, *B, *v, *gains;
    double* rtot;  // chunk totals of the long-horizon rollout of the linear models
};

// The potentials come last, so that the cached gains sit at an offset that
// does not depend on M.
static SolveBufs carve_solve(Carver& cv, int T, int d, int n, int m, int M) {
    SolveBufs b{};
    b.x = cv.take<float>((size_t)T * d);
    b.a = cv.take<float>((size_t)T * d);
    b.abar = cv.take<double>((size_t)T * n);
    b.A = cv.take<double>((size_t)T * n * n);
    b.B = cv.take<double>((size_t)T * n * m);
    b.v = cv.take<double>((size_t)T * m);
    b.gains = cv.take<double>(lqr_gain_doubles(T, n, m));
    b.rtot = cv.take<double>(rollout_scratch_doubles(T));
    b.scal = cv.take<float>(16);
    b.f = cv.take<float>((size_t)T);
    b.p = cv.take<float>((size_t)T);
    b.g = cv.take<float>((size_t)(M > 0 ? M : 1));
    return b;
}

size_t solve_buffers_bytes(int T, int d, int n, int m, int M) {
    Carver cv(nullptr);
    carve_solve(cv, T, d, n, m, M);
    return round_up(cv.off, 256);
}

void drop_solve_graph(cov_ctx* ctx) {
    if (ctx->solve_graph.exec) cudaGraphExecDestroy(ctx->solve_graph.exec);
    if (ctx->solve_graph.graph) cudaGraphDestroy(ctx->solve_graph.graph);
    ctx->solve_graph = cov_graph_cache{};
    clobber_ws_caches(ctx);
    for (cov_graph_cache* g : {&ctx->batch_graph, &ctx->ckpt_graph, &ctx->back_graph}) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        *g = cov_graph_cache{};
    }
}

// Enqueue `work` on `st` through a cached CUDA graph: captured (on a private
// stream) when `key` differs from the cached one, then launched.  With
// COV_OPT_USE_GRAPH = 0 the work is enqueued directly.
template <class F>
static cov_status run_cached_graph(cov_ctx* ctx, cov_graph_cache& gc, uint64_t key, cudaStream_t st, F&& work) {
    if (!ctx->use_graph) return work(st);
    if (!gc.exec || gc.key != key) {
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        if (gc.graph) cudaGraphDestroy(gc.graph);
        gc = cov_graph_cache{};
        cudaStream_t cap;
        if (cuda_failed(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) return COV_ERR_CUDA;
        if (cuda_failed(ctx, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) {
            cudaStreamDestroy(cap);
            return COV_ERR_CUDA;
        }
        const cov_status r = work(cap);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (r != COV_OK || cuda_failed(ctx, ce)) {
            if (g) cudaGraphDestroy(g);
            return r != COV_OK ? r : COV_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        if (cuda_failed(ctx, cudaGraphInstantiate(&ex, g, 0))) {
            cudaGraphDestroy(g);
            return COV_ERR_CUDA;
        }
        gc.graph = g;
        gc.exec = ex;
        gc.key = key;
    }
    return cuda_failed(ctx, cudaGraphLaunch(gc.exec, st)) ? COV_ERR_CUDA : COV_OK;
}

void destroy_stream_pool(cov_ctx* ctx) {
    for (cudaStream_t s : ctx->pool) cudaStreamDestroy(s);
    ctx->pool.clear();
}

// x_i = first d components of s_{i+1} (FP32 coverage coordinates).
__global__ void extract_kernel(const double* __restrict__ s, int T, int n, int d, float* __restrict__ x) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    for (int k = 0; k < d; ++k) x[(size_t)i * d + k] = (float)s[(size_t)(i + 1) * n + k];
}

// abar_t = P' a_t: the field on the coverage coordinates, zero elsewhere.
__global__ void lift_kernel(const float* __restrict__ a, int T, int n, int d, double* __restrict__ abar) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    for (int r = 0; r < n; ++r) abar[(size_t)i * n + r] = r < d ? (double)a[(size_t)i * d + r] : 0.0;
}

static uint64_t fnv(const void* p, size_t n, uint64_t h) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

// Identity of the cached time-invariant gains (and of A, B beside them in the
// solve buffers at the start of the workspace).
static uint64_t lti_gains_key(const cov_problem* P, const void* ws) {
    uint64_t gk = 88172645463325252ull;
    gk = fnv(&P->model, sizeof(int), gk);
    gk = fnv(&P->T, sizeof(int), gk);
    gk = fnv(&P->d, sizeof(int), gk);
    gk = fnv(&P->dt, sizeof(double), gk);
    gk = fnv(P->Q, sizeof(P->Q), gk);
    gk = fnv(P->R, sizeof(P->R), gk);
    gk = fnv(&ws, sizeof(ws), gk);
    return gk == 0 ? 1 : gk;
}

// Gains of a time-invariant model: computed once per (model, T, d, dt, Q, R,
// workspace) into the solve buffers and reused by every later outer
// iteration (and by the reverse sweep).  s, u: any state and control.
static cov_status ensure_lti_gains(cov_ctx* ctx, const cov_problem* P, int n, int m, const SolveBufs& b,
                                   const double* s, const double* u, cudaStream_t st) {
    const uint64_t gk = lti_gains_key(P, ctx->ws);
    if (ctx->gains_key == gk) return COV_OK;
    cov_status r = linearize_launch(ctx, P->model, s, u, P->T, P->dt, b.A, b.B, st);
    if (r != COV_OK) return r;
    r = lqr_riccati(ctx, n, m, b.A, b.B, P->Q, P->R, P->T, b.gains, st);
    if (r != COV_OK) return r;
    ctx->gains_key = gk;
    return COV_OK;
}

static cov_status validate(const cov_problem* P, int* n, int* m) {
    if (!P || model_dims(P->model, n, m) != 0) return COV_ERR_INVALID_ARG;
    if (P->T < 1 || !isfinite(P->dt) || !isfinite(P->eta) || P->d < 1 || P->d > std::min(*n, COV_MAX_D))
        return COV_ERR_INVALID_ARG;
    for (int r = 0; r < *n; ++r)
        if (!isfinite(P->s0[r])) return COV_ERR_INVALID_ARG;
    if (P->warm != 0 && P->warm != 1) return COV_ERR_INVALID_ARG;
    if (P->field == COV_FIELD_SINKHORN) {
        if (!P->y || P->M < 1 || !(P->eps > 0.f) || P->n_iter < 0) return COV_ERR_INVALID_ARG;
        if (P->eps_start > P->eps &&
            (!isfinite(P->eps_start) || !(P->eps_decay > 0.f) || !(P->eps_decay < 1.f)))
            return COV_ERR_INVALID_ARG;
    } else if (P->field == COV_FIELD_SVGD) {
        GmmParams G;
        if (!(P->h > 0.f)) return COV_ERR_INVALID_ARG;
        if (P->density) {
            if (P->d != 2 || P->density_h < 2 || P->density_w < 2) return COV_ERR_INVALID_ARG;
        } else if (make_gmm_params(&P->gmm, P->d, &G) != COV_OK) {
            return COV_ERR_INVALID_ARG;
        }
    } else {
        return COV_ERR_INVALID_ARG;
    }
    return COV_OK;
}

// The single integrator's fused LQR step + update + rollout for short
// horizons (build flag -DCOV_FUSED_SINGLE=0 takes the separate kernels).
#ifndef COV_FUSED_SINGLE
#define COV_FUSED_SINGLE 1
#endif

// Enqueue one outer iteration on `st`.
static cov_status enqueue_iteration(cov_ctx* ctx, const cov_problem* P, int n, int m, const SolveBufs& b, void* rest,
                                    size_t rest_bytes, double* u, double* s, cudaStream_t st) {
    const int T = P->T, d = P->d;
    const int nb = (T + 255) / 256;
    cov_status r = COV_ERR_UNSUPPORTED;
    if (P->field == COV_FIELD_SVGD && !P->density) {
        // short trajectories: the Stein field straight from the states s_1 .. s_T
        r = svgd_field_small(ctx, s + n, true, n, T, d, nullptr, &P->gmm, P->h, b.a, st);
        if (r != COV_OK && r != COV_ERR_UNSUPPORTED) return r;
    }
    if (r == COV_ERR_UNSUPPORTED) {
        launch_pdl(extract_kernel, dim3(nb), dim3(256), 0, st, s, T, n, d, b.x);
        if (P->field == COV_FIELD_SINKHORN) {
            const bool warm = P->warm == 1;
            r = sinkhorn_field_ws(ctx, rest, rest_bytes, b.x, d, T, P->y, P->b, P->M, d, P->eps, P->n_iter,
                                  warm ? COV_WARM_START : 0, warm ? b.f : nullptr, warm ? b.g : nullptr,
                                  warm ? b.p : nullptr, b.a, st, b.scal, P->eps_start, P->eps_decay);
        } else if (P->density) {
            // the score of the density reference, then the field (b.abar is
            // free until the lift below: the score is kept there in FP32)
            float* score = reinterpret_cast<float*>(b.abar);
            r = density_score_launch(ctx, P->density, P->density_h, P->density_w, b.x, d, T, score, st);
            if (r == COV_OK) r = svgd_field_ws(ctx, rest, rest_bytes, b.x, d, T, d, score, nullptr, P->h, b.a, st);
        } else {
            r = svgd_field_ws(ctx, rest, rest_bytes, b.x, d, T, d, nullptr, &P->gmm, P->h, b.a, st);
        }
        if (r != COV_OK) return r;
    }
    if (COV_FUSED_SINGLE && P->model == COV_SINGLE_INT) {
        // short horizons: LQR step, control update and rollout in one launch
        r = lqr_step_single_int(ctx, b.B, b.gains, P->Q, b.a, d, T, b.v, P->eta, P->dt, P->s0, u, s, st);
        if (r != COV_ERR_UNSUPPORTED) return r;
    }
    launch_pdl(lift_kernel, dim3(nb), dim3(256), 0, st, b.a, T, n, d, b.abar);
    if (!model_is_lti(P->model)) {
        r = linearize_launch(ctx, P->model, s, u, T, P->dt, b.A, b.B, st);
        if (r != COV_OK) return r;
        r = lqr_riccati(ctx, n, m, b.A, b.B, P->Q, P->R, T, b.gains, st);
        if (r != COV_OK) return r;
    }
    r = lqr_affine(ctx, rest, rest_bytes, n, m, b.B, b.gains, P->Q, b.abar, T, b.v, nullptr, st);
    if (r != COV_OK) return r;
    r = update_rollout(ctx, P->model, P->s0, u, b.v, P->eta, T, P->dt, s, st, b.rtot);
    if (r != COV_OK) return r;
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

}  // namespace cov

namespace cov {
static cov_status solve_impl(cov_ctx* ctx, const cov_problem* prob, int n_outer, double* u, double* s_out,
                             cudaStream_t stream, bool initial_rollout, double* s_hist = nullptr);
}

extern "C" cov_status cov_solve(cov_ctx* ctx, const cov_problem* prob, int n_outer, double* u, double* s_out,
                                cov_stream_t stream) {
    return cov::solve_impl(ctx, prob, n_outer, u, s_out, (cudaStream_t)stream, true);
}

extern "C" cov_status cov_solve_continue(cov_ctx* ctx, const cov_problem* prob, int n_outer, double* u, double* s,
                                         cov_stream_t stream) {
    return cov::solve_impl(ctx, prob, n_outer, u, s, (cudaStream_t)stream, false);
}

static cov_status cov::solve_impl(cov_ctx* ctx, const cov_problem* prob, int n_outer, double* u, double* s_out,
                                  cudaStream_t stream, bool initial_rollout, double* s_hist) {
    using namespace cov;
    int n, m;
    if (!ctx || !u || !s_out || n_outer < 0) return COV_ERR_INVALID_ARG;
    cov_status r = validate(prob, &n, &m);
    if (r != COV_OK) return r;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cudaStream_t st = stream;
    Carver cv(ctx->ws);
    SolveBufs b = carve_solve(cv, prob->T, prob->d, n, m, prob_M(prob));
    const size_t used = round_up(cv.off, 256);
    if (!ctx->ws || used > ctx->ws_bytes) return COV_ERR_WORKSPACE;
    void* rest = static_cast<char*>(ctx->ws) + used;
    const size_t rest_bytes = ctx->ws_bytes - used;
    ctx->tape_key = 0;  // the scratch below overwrites forward records

    // warm-started potentials: a fresh solve starts cold (zero potentials
    // with the warm flag are exactly the cold start); a continuation keeps
    // them while nothing else has run on the context
    const bool warm = prob->field == COV_FIELD_SINKHORN && prob->warm == 1;
    uint64_t pk = 0;
    if (warm) {
        pk = 9650029242287828579ull;
        pk = fnv(prob, sizeof(cov_problem), pk);
        const void* ptrs[3] = {u, s_out, ctx->ws};
        pk = fnv(ptrs, sizeof(ptrs), pk);
        if (initial_rollout || ctx->pot_key != pk) {
            ctx->pot_key = 0;
            if (cuda_failed(ctx, cudaMemsetAsync(b.f, 0, sizeof(float) * prob->T, st)) ||
                cuda_failed(ctx, cudaMemsetAsync(b.p, 0, sizeof(float) * prob->T, st)) ||
                cuda_failed(ctx, cudaMemsetAsync(b.g, 0, sizeof(float) * prob->M, st)))
                return COV_ERR_CUDA;
        }
    }

    // initial trajectory from s0 and the given controls
    if (initial_rollout) {
        r = update_rollout(ctx, prob->model, prob->s0, u, nullptr, 0.0, prob->T, prob->dt, s_out, st, b.rtot);
        if (r != COV_OK) return r;
    }
    if (n_outer == 0) return COV_OK;
    // the reference set is fixed during a solve: its centre and weight sum
    // are computed once per call
    if (prob->field == COV_FIELD_SINKHORN) sinkhorn_reference_stats(prob->y, prob->M, prob->d, prob->b, b.scal, st);

    if (model_is_lti(prob->model)) {
        r = ensure_lti_gains(ctx, prob, n, m, b, s_out, u, st);
        if (r != COV_OK) return r;
    }

    // checkpoint k: the trajectory entering outer iteration k
    const size_t ss_bytes = sizeof(double) * (size_t)(prob->T + 1) * n;
    auto checkpoint = [&](int k) {
        return s_hist ? cuda_failed(ctx, cudaMemcpyAsync(s_hist + (size_t)k * (prob->T + 1) * n, s_out, ss_bytes,
                                                         cudaMemcpyDeviceToDevice, st))
                      : false;
    };
    if (!ctx->use_graph) {
        for (int k = 0; k < n_outer; ++k) {
            if (checkpoint(k)) return COV_ERR_CUDA;
            r = enqueue_iteration(ctx, prob, n, m, b, rest, rest_bytes, u, s_out, st);
            if (r != COV_OK) return r;
        }
        if (warm) ctx->pot_key = pk;
        return COV_OK;
    }
    uint64_t key = 1469598103934665603ull;
    key = fnv(prob, sizeof(cov_problem), key);
    if (prob->field == COV_FIELD_SVGD) {
        key = fnv(prob->gmm.w, sizeof(float) * prob->gmm.K, key);
        key = fnv(prob->gmm.mu, sizeof(float) * prob->gmm.K * prob->d, key);
        key = fnv(prob->gmm.sigma, sizeof(float) * prob->gmm.K, key);
    }
    const void* ptrs[3] = {u, s_out, ctx->ws};
    key = fnv(ptrs, sizeof(ptrs), key);
    if (!ctx->solve_graph.exec || ctx->solve_graph.key != key) {
        drop_solve_graph(ctx);
        cudaStream_t cap;
        if (cuda_failed(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) return COV_ERR_CUDA;
        cudaGraph_t g = nullptr;
        if (cuda_failed(ctx, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) {
            cudaStreamDestroy(cap);
            return COV_ERR_CUDA;
        }
        const cov_status er = enqueue_iteration(ctx, prob, n, m, b, rest, rest_bytes, u, s_out, cap);
        const cudaError_t ce = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (er != COV_OK) {
            if (g) cudaGraphDestroy(g);
            return er;
        }
        if (cuda_failed(ctx, ce)) return COV_ERR_CUDA;
        cudaGraphExec_t ex = nullptr;
        if (cuda_failed(ctx, cudaGraphInstantiate(&ex, g, 0))) {
            cudaGraphDestroy(g);
            return COV_ERR_CUDA;
        }
        ctx->solve_graph.graph = g;
        ctx->solve_graph.exec = ex;
        ctx->solve_graph.key = key;
    }
    for (int k = 0; k < n_outer; ++k) {
        if (checkpoint(k)) return COV_ERR_CUDA;
        if (cuda_failed(ctx, cudaGraphLaunch(ctx->solve_graph.exec, st))) return COV_ERR_CUDA;
    }
    if (warm) ctx->pot_key = pk;
    return COV_OK;
}

// ---------------------------------------------------------------------------
// Batched solve: many independent problems, one CUDA graph per outer
// iteration.  Each problem owns a contiguous region of the workspace (its
// solve buffers, then the field / LQR scratch).  One outer iteration of every
// problem is captured as an independent branch of a single graph (branches
// forked over a pool of streams during capture), so one graph launch
// advances all problems and the GPU interleaves their kernels.
// ---------------------------------------------------------------------------
namespace cov {

// Streams the batch's branches are captured on (problems p, p + K, ... of
// one stream run one after another; build flag -DCOV_POOL_STREAMS=K).
#ifndef COV_POOL_STREAMS
#define COV_POOL_STREAMS 64
#endif
static constexpr int kPoolStreams = COV_POOL_STREAMS;

static size_t problem_ws_bytes(const cov_problem* P, int n, int m) {
    const size_t solve = solve_buffers_bytes(P->T, P->d, n, m, prob_M(P));
    const size_t field =
        P->field == COV_FIELD_SINKHORN ? sinkhorn_ws_bytes(P->T, P->M, P->d) : svgd_ws_bytes(P->T, P->d);
    const size_t lqr = lqr_ws_bytes(P->T, n, m);
    return round_up(solve + std::max(field, lqr) + 4096, 256);
}

static cov_status ensure_pool(cov_ctx* ctx, int k) {
    while ((int)ctx->pool.size() < k) {
        cudaStream_t s;
        if (cuda_failed(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking))) return COV_ERR_CUDA;
        ctx->pool.push_back(s);
    }
    return COV_OK;
}

// Make each of streams[0..k) wait for the work so far on `from`.
static cov_status fork_streams(cov_ctx* ctx, cudaStream_t from, const std::vector<cudaStream_t>& to, int k) {
    cudaEvent_t e;
    if (cuda_failed(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming))) return COV_ERR_CUDA;
    cov_status r = COV_OK;
    if (cuda_failed(ctx, cudaEventRecord(e, from))) r = COV_ERR_CUDA;
    for (int i = 0; i < k && r == COV_OK; ++i)
        if (cuda_failed(ctx, cudaStreamWaitEvent(to[i], e, 0))) r = COV_ERR_CUDA;
    cudaEventDestroy(e);
    return r;
}

// Make `into` wait for the work so far on streams[0..k).
static cov_status join_streams(cov_ctx* ctx, const std::vector<cudaStream_t>& from, int k, cudaStream_t into) {
    for (int i = 0; i < k; ++i) {
        cudaEvent_t e;
        if (cuda_failed(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming))) return COV_ERR_CUDA;
        const bool bad = cuda_failed(ctx, cudaEventRecord(e, from[i])) || cuda_failed(ctx, cudaStreamWaitEvent(into, e, 0));
        cudaEventDestroy(e);
        if (bad) return COV_ERR_CUDA;
    }
    return COV_OK;
}

}  // namespace cov

extern "C" size_t cov_workspace_size_batched(const cov_problem* probs, int n_probs) {
    if (!probs || n_probs < 1) return 0;
    size_t total = 0;
    for (int p = 0; p < n_probs; ++p) {
        int n, m;
        if (cov::validate(&probs[p], &n, &m) != COV_OK) return 0;
        total += cov::problem_ws_bytes(&probs[p], n, m);
    }
    return total + 4096;
}

extern "C" cov_status cov_solve_batched(cov_ctx* ctx, const cov_problem* probs, int n_probs, int n_outer,
                                        double* const* u, double* const* s_out, cov_stream_t stream) {
    using namespace cov;
    if (!ctx || !probs || n_probs < 1 || n_outer < 0 || !u || !s_out) return COV_ERR_INVALID_ARG;
    std::vector<int> nn(n_probs), mm(n_probs);
    std::vector<size_t> off(n_probs);
    size_t total = 0;
    for (int p = 0; p < n_probs; ++p) {
        if (!u[p] || !s_out[p]) return COV_ERR_INVALID_ARG;
        const cov_status r = validate(&probs[p], &nn[p], &mm[p]);
        if (r != COV_OK) return r;
        off[p] = total;
        total += problem_ws_bytes(&probs[p], nn[p], mm[p]);
    }
    if (!ctx->ws || total > ctx->ws_bytes) return COV_ERR_WORKSPACE;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    clobber_ws_caches(ctx);  // the problem regions overlap what cov_solve cached
    cudaStream_t st = (cudaStream_t)stream;
    const int K = std::min(n_probs, kPoolStreams);
    if (ensure_pool(ctx, K) != COV_OK) return COV_ERR_CUDA;

    std::vector<SolveBufs> bufs(n_probs);
    std::vector<void*> rest(n_probs);
    std::vector<size_t> rest_bytes(n_probs);
    for (int p = 0; p < n_probs; ++p) {
        char* base = static_cast<char*>(ctx->ws) + off[p];
        Carver cv(base);
        bufs[p] = carve_solve(cv, probs[p].T, probs[p].d, nn[p], mm[p], prob_M(&probs[p]));
        const size_t used = round_up(cv.off, 256);
        rest[p] = base + used;
        rest_bytes[p] = problem_ws_bytes(&probs[p], nn[p], mm[p]) - used;
    }

    // set-up of every problem, spread over the pool: initial rollout, the
    // reference statistics, and the Riccati gains of time-invariant models
    cov_status r = fork_streams(ctx, st, ctx->pool, K);
    if (r != COV_OK) return r;
    for (int p = 0; p < n_probs && r == COV_OK; ++p) {
        const cov_problem* P = &probs[p];
        cudaStream_t sp = ctx->pool[p % K];
        r = update_rollout(ctx, P->model, P->s0, u[p], nullptr, 0.0, P->T, P->dt, s_out[p], sp, bufs[p].rtot);
        if (r != COV_OK || n_outer == 0) continue;
        if (P->field == COV_FIELD_SINKHORN) {
            sinkhorn_reference_stats(P->y, P->M, P->d, P->b, bufs[p].scal, sp);
            if (P->warm == 1 &&
                (cuda_failed(ctx, cudaMemsetAsync(bufs[p].f, 0, sizeof(float) * P->T, sp)) ||
                 cuda_failed(ctx, cudaMemsetAsync(bufs[p].p, 0, sizeof(float) * P->T, sp)) ||
                 cuda_failed(ctx, cudaMemsetAsync(bufs[p].g, 0, sizeof(float) * P->M, sp))))
                r = COV_ERR_CUDA;
        }
        if (model_is_lti(P->model)) {
            r = linearize_launch(ctx, P->model, s_out[p], u[p], P->T, P->dt, bufs[p].A, bufs[p].B, sp);
            if (r == COV_OK) r = lqr_riccati(ctx, nn[p], mm[p], bufs[p].A, bufs[p].B, P->Q, P->R, P->T,
                                             bufs[p].gains, sp);
        }
    }
    if (r != COV_OK) return r;
    r = join_streams(ctx, ctx->pool, K, st);
    if (r != COV_OK || n_outer == 0) return r;

    if (!ctx->use_graph) {
        for (int k = 0; k < n_outer && r == COV_OK; ++k) {
            r = fork_streams(ctx, st, ctx->pool, K);
            ctx->plan_share = ctx->batch_share;
            for (int p = 0; p < n_probs && r == COV_OK; ++p)
                r = enqueue_iteration(ctx, &probs[p], nn[p], mm[p], bufs[p], rest[p], rest_bytes[p], u[p], s_out[p],
                                      ctx->pool[p % K]);
            ctx->plan_share = 100;
            if (r == COV_OK) r = join_streams(ctx, ctx->pool, K, st);
        }
        return r;
    }

    uint64_t key = 1469598103934665603ull;
    for (int p = 0; p < n_probs; ++p) {
        key = fnv(&probs[p], sizeof(cov_problem), key);
        if (probs[p].field == COV_FIELD_SVGD) {
            key = fnv(probs[p].gmm.w, sizeof(float) * probs[p].gmm.K, key);
            key = fnv(probs[p].gmm.mu, sizeof(float) * probs[p].gmm.K * probs[p].d, key);
            key = fnv(probs[p].gmm.sigma, sizeof(float) * probs[p].gmm.K, key);
        }
        const void* ptrs[2] = {u[p], s_out[p]};
        key = fnv(ptrs, sizeof(ptrs), key);
    }
    const void* wsp = ctx->ws;
    key = fnv(&wsp, sizeof(wsp), key);
    if (!ctx->batch_graph.exec || ctx->batch_graph.key != key) {
        if (ctx->batch_graph.exec) cudaGraphExecDestroy(ctx->batch_graph.exec);
        if (ctx->batch_graph.graph) cudaGraphDestroy(ctx->batch_graph.graph);
        ctx->batch_graph = cov_graph_cache{};
        cudaStream_t cap;
        if (cuda_failed(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) return COV_ERR_CUDA;
        if (cuda_failed(ctx, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) {
            cudaStreamDestroy(cap);
            return COV_ERR_CUDA;
        }
        r = fork_streams(ctx, cap, ctx->pool, K);
        ctx->plan_share = ctx->batch_share;  // the problems' launches run side by side
        for (int p = 0; p < n_probs && r == COV_OK; ++p)
            r = enqueue_iteration(ctx, &probs[p], nn[p], mm[p], bufs[p], rest[p], rest_bytes[p], u[p], s_out[p],
                                  ctx->pool[p % K]);
        ctx->plan_share = 100;
        if (r == COV_OK) r = join_streams(ctx, ctx->pool, K, cap);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (r != COV_OK || cuda_failed(ctx, ce)) {
            if (g) cudaGraphDestroy(g);
            return r != COV_OK ? r : COV_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        if (cuda_failed(ctx, cudaGraphInstantiate(&ex, g, 0))) {
            cudaGraphDestroy(g);
            return COV_ERR_CUDA;
        }
        ctx->batch_graph.graph = g;
        ctx->batch_graph.exec = ex;
        ctx->batch_graph.key = key;
    }
    for (int k = 0; k < n_outer; ++k)
        if (cuda_failed(ctx, cudaGraphLaunch(ctx->batch_graph.exec, st))) return COV_ERR_CUDA;
    return COV_OK;
}

// ---------------------------------------------------------------------------
// Gradient through the outer iteration (reverse mode, checkpointed).  For a
// time-invariant model A, B do not depend on the trajectory, so v^k depends
// on the previous trajectory s^{k-1} only through the field, and
//   ubar^K = rollout_vjp(sbar_K),
//   k = K..1:  abar_bar = lqr_vjp(eta ubar^k);
//              (xbar, ybar, bbar) += field_vjp(x^{k-1}; abar_bar);
//              ubar^{k-1} = ubar^k + rollout_vjp(lift(xbar)),
//   s0bar = sum of the rollout adjoints' lambda_0, u0bar = ubar^0.
// The trajectories s^0..s^{K-1} are the checkpoints (given, or rebuilt by
// replaying the forward from u0).  The field VJP needs the Sinkhorn
// iterations of each outer iteration: a taped forward keeps their records
// in the workspace (HBM is plentiful: (2 + d)(n_iter + 2)(T + M) floats per
// outer iteration), otherwise they are recomputed from the checkpoint.
//
// Workspace layout (shared by the taped forward and the backward):
//   [solve buffers][records: K slots][split buffers][backward buffers][rest]
// with the records and split buffers present in mode 2 only.
// ---------------------------------------------------------------------------
namespace cov {
size_t lqr_adj_ws_bytes(int T, int n, int m);
size_t lqr_ws_bytes(int T, int n, int m);
cov_status lqr_vjp_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, int n, int m, const double* B, const double* gains,
                      const double* Q, const double* vbar, int T, double* abar_bar, cudaStream_t stream);
cov_status rollout_vjp_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, int n, int m, const double* A, const double* B,
                          const double* sbar, int T, double* ubar, double* s0bar, cudaStream_t stream);

enum BackMode { BM_GIVEN = 0, BM_REPLAY = 1, BM_TAPED = 2 };

struct BackBufs {
    float *xbar, *abf;
    double *abb, *sbar, *ubar, *ub2, *vbar, *lam0, *u, *hist;
};

struct BackLayout {
    SolveBufs sb;
    char* tape0;       // record slot k at tape0 + k * tape_stride
    size_t tape_stride;
    float* split;      // split buffers shared by the records' passes
    BackBufs bb;
    char* rest;
    size_t rest_bytes;
    size_t needed;     // total bytes the mode needs
};

static BackBufs carve_back(Carver& cv, int T, int d, int n, int m, int n_hist) {
    BackBufs b{};
    b.xbar = cv.take<float>((size_t)T * d);
    b.abf = cv.take<float>((size_t)T * d);
    b.abb = cv.take<double>((size_t)T * n);
    b.sbar = cv.take<double>((size_t)(T + 1) * n);
    b.ubar = cv.take<double>((size_t)T * m);
    b.ub2 = cv.take<double>((size_t)T * m);
    b.vbar = cv.take<double>((size_t)T * m);
    b.lam0 = cv.take<double>(COV_MAX_N);
    b.u = cv.take<double>((size_t)T * m);
    b.hist = n_hist > 0 ? cv.take<double>((size_t)n_hist * (T + 1) * n) : nullptr;
    return b;
}

static bool backward_supported(const cov_problem* P) {
    return P->field == COV_FIELD_SINKHORN && model_is_lti(P->model) && P->d <= 3 && P->warm == 0 &&
           !(P->eps_start > P->eps);
}
// Stein field with a mixture reference on a time-invariant model.
static bool backward_svgd_supported(const cov_problem* P) {
    return P->field == COV_FIELD_SVGD && model_is_lti(P->model) && !P->density;
}

// ws == nullptr only measures (L->needed).
static void carve_layout(void* ws, size_t ws_bytes, const cov_problem* P, int n, int m, int K, int mode,
                         BackLayout* L) {
    const int T = P->T, d = P->d;
    Carver cv(ws);
    *L = BackLayout{};
    L->sb = carve_solve(cv, T, d, n, m, prob_M(P));
    if (mode == BM_TAPED) {
        L->tape_stride = round_up(sinkhorn_tape_bytes(T, P->M, d, P->n_iter, false), 256);
        L->tape0 = cv.take<char>(L->tape_stride * (size_t)K);
        L->split = reinterpret_cast<float*>(cv.take<char>(sinkhorn_split_bytes(T, P->M, d)));
    }
    L->bb = carve_back(cv, T, d, n, m, mode == BM_REPLAY ? K : 0);
    const size_t used = round_up(cv.off, 256);
    size_t rest = std::max(lqr_adj_ws_bytes(T, n, m), lqr_ws_bytes(T, n, m));
    if (P->field == COV_FIELD_SVGD) {
        rest = std::max(rest, svgd_vjp_ws_bytes(T, d, P->gmm.K, 1024));
        if (mode == BM_REPLAY) rest = std::max(rest, svgd_ws_bytes(T, d));
    } else {
        rest = std::max(rest, mode == BM_TAPED ? sinkhorn_vjp_bytes_given(T, P->M, d)
                                               : sinkhorn_vjp_bytes(T, P->M, d, P->n_iter));
        if (mode == BM_REPLAY) rest = std::max(rest, sinkhorn_ws_bytes(T, P->M, d));
    }
    L->needed = used + rest + 4096;
    L->rest = ws ? static_cast<char*>(ws) + used : nullptr;
    L->rest_bytes = ws_bytes > used ? ws_bytes - used : 0;
}

static uint64_t tape_key_of(const cov_problem* P, int K, const double* s_hist, const cov_ctx* ctx) {
    uint64_t k = 7809847782465536322ull;
    k = fnv(P, sizeof(cov_problem), k);
    k = fnv(&K, sizeof(K), k);
    k = fnv(&s_hist, sizeof(s_hist), k);
    k = fnv(&ctx->ws, sizeof(ctx->ws), k);
    k = fnv(&ctx->ws_bytes, sizeof(ctx->ws_bytes), k);
    return k == 0 ? 1 : k;
}

// vbar = eta ubar
__global__ void back_scale_kernel(const double* __restrict__ ubar, double eta, int N, double* __restrict__ vbar) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) vbar[i] = eta * ubar[i];
}
// abf = the coverage components of abar_bar, in FP32
__global__ void narrow_kernel(const double* __restrict__ abb, int T, int n, int d, float* __restrict__ abf) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    for (int k = 0; k < d; ++k) abf[(size_t)i * d + k] = (float)abb[(size_t)i * n + k];
}
// sbar = the sample adjoint lifted to the trajectory (s_0 does not move)
__global__ void lift_bar_kernel(const float* __restrict__ xbar, int T, int n, int d, double* __restrict__ sbar) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > T) return;
    for (int r = 0; r < n; ++r)
        sbar[(size_t)i * n + r] = (i >= 1 && r < d) ? (double)xbar[(size_t)(i - 1) * d + r] : 0.0;
}
// ubar += ub2; s0bar += lam0
__global__ void back_accum_kernel(double* __restrict__ ubar, const double* __restrict__ ub2, int N,
                                  double* __restrict__ s0bar, const double* __restrict__ lam0, int n) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) ubar[i] += ub2[i];
    if (i < n) s0bar[i] += lam0[i];
}

// Taped forward: cov_solve from u (initial rollout included) that keeps the
// checkpoints s_hist[k] and, per outer iteration, the record of its field's
// Sinkhorn iterations.
static cov_status solve_taped(cov_ctx* ctx, const cov_problem* prob, int K, double* u, double* s_out,
                              double* s_hist, cudaStream_t st) {
    int n, m;
    cov_status r = validate(prob, &n, &m);
    if (r != COV_OK) return r;
    if (!backward_supported(prob)) return COV_ERR_UNSUPPORTED;
    BackLayout L;
    carve_layout(nullptr, 0, prob, n, m, K, BM_TAPED, &L);
    if (!ctx->ws || L.needed > ctx->ws_bytes) return COV_ERR_WORKSPACE;
    carve_layout(ctx->ws, ctx->ws_bytes, prob, n, m, K, BM_TAPED, &L);
    ctx->tape_key = 0;
    const int T = prob->T, d = prob->d;
    const size_t ss = (size_t)(T + 1) * n;
    const int nb = (T + 255) / 256;
    const SolveBufs& b = L.sb;
    if (K > 0) {
        // time-invariant gains first (host-side cache decision); A, B do not
        // read the trajectory, so s_out's current contents do not matter
        r = ensure_lti_gains(ctx, prob, n, m, b, s_out, u, st);
        if (r != COV_OK) return r;
    }
    auto work = [&](cudaStream_t ws_st) -> cov_status {
        cov_status q = update_rollout(ctx, prob->model, prob->s0, u, nullptr, 0.0, T, prob->dt, s_out, ws_st, b.rtot);
        if (q != COV_OK || K == 0) return q;
        sinkhorn_reference_stats(prob->y, prob->M, d, prob->b, b.scal, ws_st);
        ctx->tapes.assign(K, SkTape{});
        for (int k = 0; k < K; ++k) {
            if (cuda_failed(ctx, cudaMemcpyAsync(s_hist + (size_t)k * ss, s_out, sizeof(double) * ss,
                                                 cudaMemcpyDeviceToDevice, ws_st)))
                return COV_ERR_CUDA;
            launch_pdl(extract_kernel, dim3(nb), dim3(256), 0, ws_st, s_out, T, n, d, b.x);
            size_t used = 0;
            q = sinkhorn_tape_ws(ctx, L.tape0 + (size_t)k * L.tape_stride, L.tape_stride, b.x, d, T, prob->y,
                                 prob->b, prob->M, d, prob->eps, prob->n_iter, b.scal, &ctx->tapes[k], &used, ws_st,
                                 L.split, b.a);
            if (q != COV_OK) return q;
            launch_pdl(lift_kernel, dim3(nb), dim3(256), 0, ws_st, b.a, T, n, d, b.abar);
            q = lqr_affine(ctx, L.rest, L.rest_bytes, n, m, b.B, b.gains, prob->Q, b.abar, T, b.v, nullptr, ws_st);
            if (q != COV_OK) return q;
            q = update_rollout(ctx, prob->model, prob->s0, u, b.v, prob->eta, T, prob->dt, s_out, ws_st, b.rtot);
            if (q != COV_OK) return q;
        }
        return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;
    };
    uint64_t key = 5851236489572341227ull;
    key = fnv(prob, sizeof(cov_problem), key);
    key = fnv(&K, sizeof(K), key);
    const void* ptrs[5] = {u, s_out, s_hist, ctx->ws, reinterpret_cast<const void*>(ctx->ws_bytes)};
    key = fnv(ptrs, sizeof(ptrs), key);
    r = run_cached_graph(ctx, ctx->ckpt_graph, key, st, work);
    if (r != COV_OK) return r;
    if (K > 0) ctx->tape_key = tape_key_of(prob, K, s_hist, ctx);
    return COV_OK;
}

}  // namespace cov

extern "C" cov_status cov_solve_checkpointed(cov_ctx* ctx, const cov_problem* prob, int n_outer, double* u,
                                             double* s_out, double* s_hist, int flags, cov_stream_t stream) {
    if (!ctx || !u || !s_out || n_outer < 0 || (!s_hist && n_outer > 0) || (flags & ~COV_CKPT_RECORD))
        return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    if (flags & COV_CKPT_RECORD) return cov::solve_taped(ctx, prob, n_outer, u, s_out, s_hist, (cudaStream_t)stream);
    return cov::solve_impl(ctx, prob, n_outer, u, s_out, (cudaStream_t)stream, true, s_hist);
}

extern "C" size_t cov_workspace_size_backward(const cov_problem* prob, int n_outer, int mode) {
    int n, m;
    if (!prob || n_outer < 0 || mode < 0 || mode > 2 || cov::validate(prob, &n, &m) != COV_OK ||
        !(cov::backward_supported(prob) || (cov::backward_svgd_supported(prob) && mode != cov::BM_TAPED)))
        return 0;
    cov::BackLayout L;
    cov::carve_layout(nullptr, 0, prob, n, m, n_outer, mode, &L);
    return L.needed;
}

extern "C" cov_status cov_solve_backward(cov_ctx* ctx, const cov_problem* prob, int n_outer, const double* u0,
                                         const double* s_hist, const double* sbar_K, float* ybar, float* bbar,
                                         double* s0bar, double* u0bar, cov_stream_t stream) {
    using namespace cov;
    int n, m;
    if (!ctx || n_outer < 0 || !u0 || !sbar_K || !ybar || !s0bar) return COV_ERR_INVALID_ARG;
    cov_status r = validate(prob, &n, &m);
    if (r != COV_OK) return r;
    if (!backward_supported(prob)) return COV_ERR_UNSUPPORTED;
    if (prob->b && !bbar) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    const int T = prob->T, d = prob->d, K = n_outer;
    int mode = s_hist ? BM_GIVEN : BM_REPLAY;
    if (s_hist && K > 0 && ctx->tape_key == tape_key_of(prob, K, s_hist, ctx) && (int)ctx->tapes.size() == K)
        mode = BM_TAPED;
    BackLayout L;
    carve_layout(nullptr, 0, prob, n, m, K, mode, &L);
    if (!ctx->ws || L.needed > ctx->ws_bytes) return COV_ERR_WORKSPACE;
    carve_layout(ctx->ws, ctx->ws_bytes, prob, n, m, K, mode, &L);
    if (mode != BM_TAPED) ctx->tape_key = 0;  // the backward buffers overlap the record slots
    const SolveBufs& sb = L.sb;
    const BackBufs& bb = L.bb;
    void* rest = L.rest;
    const size_t rest_bytes = L.rest_bytes;
    cudaStream_t stream0 = (cudaStream_t)stream;
    const size_t ss = (size_t)(T + 1) * n;
    const int nb = (T + 256) / 256;

    // A, B (time-invariant: any state will do) and the Riccati gains, shared
    // with cov_solve's cache (same solve buffers at the start of the
    // workspace); decided on the host before the reverse sweep is enqueued
    r = ensure_lti_gains(ctx, prob, n, m, sb, sbar_K, u0, stream0);
    if (r != COV_OK) return r;
    auto work = [&](cudaStream_t st) -> cov_status {
    cov_status r = COV_OK;
    sinkhorn_reference_stats(prob->y, prob->M, d, prob->b, sb.scal, st);
    const double* hist = s_hist;
    if (mode == BM_REPLAY) {
        // rebuild the checkpoints s^0..s^{K-1} from u0
        if (cuda_failed(ctx, cudaMemcpyAsync(bb.u, u0, sizeof(double) * T * m, cudaMemcpyDeviceToDevice, st)))
            return COV_ERR_CUDA;
        if (K > 0) {
            r = update_rollout(ctx, prob->model, prob->s0, bb.u, nullptr, 0.0, T, prob->dt, bb.hist, st);
            if (r != COV_OK) return r;
        }
        hist = bb.hist;
    }
    if (mode == BM_REPLAY) {
        for (int k = 1; k < K; ++k) {
            double* sk = bb.hist + (size_t)k * ss;
            if (cuda_failed(ctx, cudaMemcpyAsync(sk, sk - ss, sizeof(double) * ss, cudaMemcpyDeviceToDevice, st)))
                return COV_ERR_CUDA;
            r = enqueue_iteration(ctx, prob, n, m, sb, rest, rest_bytes, bb.u, sk, st);
            if (r != COV_OK) return r;
        }
    }
    // final rollout adjoint
    r = rollout_vjp_ws(ctx, rest, rest_bytes, n, m, sb.A, sb.B, sbar_K, T, bb.ubar, s0bar, st);
    if (r != COV_OK) return r;
    if (K == 0) {
        if (cuda_failed(ctx, cudaMemsetAsync(ybar, 0, sizeof(float) * prob->M * d, st))) return COV_ERR_CUDA;
        if (bbar && cuda_failed(ctx, cudaMemsetAsync(bbar, 0, sizeof(float) * prob->M, st))) return COV_ERR_CUDA;
    }
    const int Tm = T * m;
    for (int k = K; k >= 1; --k) {
        launch_pdl(back_scale_kernel, dim3((Tm + 255) / 256), dim3(256), 0, st, bb.ubar, prob->eta, Tm, bb.vbar);
        r = lqr_vjp_ws(ctx, rest, rest_bytes, n, m, sb.B, sb.gains, prob->Q, bb.vbar, T, bb.abb, st);
        if (r != COV_OK) return r;
        launch_pdl(narrow_kernel, dim3(nb), dim3(256), 0, st, bb.abb, T, n, d, bb.abf);
        if (mode != BM_TAPED) launch_pdl(extract_kernel, dim3(nb), dim3(256), 0, st, hist + (size_t)(k - 1) * ss, T, n, d, sb.x);
        r = sinkhorn_vjp_ws(ctx, rest, rest_bytes, sb.x, d, T, prob->y, prob->b, prob->M, d, prob->eps,
                            prob->n_iter, sb.scal, bb.abf, d, bb.xbar, d, ybar, prob->b ? bbar : nullptr,
                            k != K ? 1 : 0, st, mode == BM_TAPED ? &ctx->tapes[k - 1] : nullptr);
        if (r != COV_OK) return r;
        launch_pdl(lift_bar_kernel, dim3(nb), dim3(256), 0, st, bb.xbar, T, n, d, bb.sbar);
        r = rollout_vjp_ws(ctx, rest, rest_bytes, n, m, sb.A, sb.B, bb.sbar, T, bb.ub2, bb.lam0, st);
        if (r != COV_OK) return r;
        launch_pdl(back_accum_kernel, dim3((Tm + 255) / 256), dim3(256), 0, st, bb.ubar, bb.ub2, Tm, s0bar, bb.lam0, n);
    }
    if (u0bar && cuda_failed(ctx, cudaMemcpyAsync(u0bar, bb.ubar, sizeof(double) * Tm, cudaMemcpyDeviceToDevice, st)))
        return COV_ERR_CUDA;
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
    };
    uint64_t key = 2305843009213693951ull;
    key = fnv(prob, sizeof(cov_problem), key);
    key = fnv(&K, sizeof(K), key);
    key = fnv(&mode, sizeof(mode), key);
    const void* ptrs[9] = {u0, s_hist, sbar_K, ybar, bbar, s0bar, u0bar, ctx->ws,
                           reinterpret_cast<const void*>(ctx->ws_bytes)};
    key = fnv(ptrs, sizeof(ptrs), key);
    return run_cached_graph(ctx, ctx->back_graph, key, stream0, work);
}

// Gradient through K outer iterations of a Stein-field solve with a mixture
// reference (time-invariant model): the reverse sweep of cov_solve_backward
// with the Stein field's reverse mode in place of the Sinkhorn one; the
// mixture gradients of every outer iteration are summed.
extern "C" cov_status cov_solve_backward_svgd(cov_ctx* ctx, const cov_problem* prob, int n_outer, const double* u0,
                                              const double* s_hist, const double* sbar_K, float* wbar, float* mubar,
                                              float* sigmabar, double* s0bar, double* u0bar, cov_stream_t stream) {
    using namespace cov;
    int n, m;
    if (!ctx || n_outer < 0 || !u0 || !sbar_K || !s0bar) return COV_ERR_INVALID_ARG;
    cov_status r = validate(prob, &n, &m);
    if (r != COV_OK) return r;
    if (!backward_svgd_supported(prob)) return COV_ERR_UNSUPPORTED;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    const int T = prob->T, d = prob->d, K = n_outer, KG = prob->gmm.K;
    const int mode = s_hist ? BM_GIVEN : BM_REPLAY;
    BackLayout L;
    carve_layout(nullptr, 0, prob, n, m, K, mode, &L);
    if (!ctx->ws || L.needed > ctx->ws_bytes) return COV_ERR_WORKSPACE;
    carve_layout(ctx->ws, ctx->ws_bytes, prob, n, m, K, mode, &L);
    ctx->tape_key = 0;  // the backward buffers overlap the record slots
    const SolveBufs& sb = L.sb;
    const BackBufs& bb = L.bb;
    void* rest = L.rest;
    const size_t rest_bytes = L.rest_bytes;
    cudaStream_t stream0 = (cudaStream_t)stream;
    const size_t ss = (size_t)(T + 1) * n;
    const int nb = (T + 256) / 256;
    r = ensure_lti_gains(ctx, prob, n, m, sb, sbar_K, u0, stream0);
    if (r != COV_OK) return r;
    auto work = [&](cudaStream_t st) -> cov_status {
        cov_status q = COV_OK;
        const double* hist = s_hist;
        if (mode == BM_REPLAY) {
            // rebuild the checkpoints s^0..s^{K-1} from u0
            if (cuda_failed(ctx, cudaMemcpyAsync(bb.u, u0, sizeof(double) * T * m, cudaMemcpyDeviceToDevice, st)))
                return COV_ERR_CUDA;
            if (K > 0) {
                q = update_rollout(ctx, prob->model, prob->s0, bb.u, nullptr, 0.0, T, prob->dt, bb.hist, st);
                if (q != COV_OK) return q;
            }
            for (int k = 1; k < K; ++k) {
                double* sk = bb.hist + (size_t)k * ss;
                if (cuda_failed(ctx, cudaMemcpyAsync(sk, sk - ss, sizeof(double) * ss, cudaMemcpyDeviceToDevice, st)))
                    return COV_ERR_CUDA;
                q = enqueue_iteration(ctx, prob, n, m, sb, rest, rest_bytes, bb.u, sk, st);
                if (q != COV_OK) return q;
            }
            hist = bb.hist;
        }
        q = rollout_vjp_ws(ctx, rest, rest_bytes, n, m, sb.A, sb.B, sbar_K, T, bb.ubar, s0bar, st);
        if (q != COV_OK) return q;
        if (K == 0) {
            if ((wbar && cuda_failed(ctx, cudaMemsetAsync(wbar, 0, sizeof(float) * KG, st))) ||
                (mubar && cuda_failed(ctx, cudaMemsetAsync(mubar, 0, sizeof(float) * KG * d, st))) ||
                (sigmabar && cuda_failed(ctx, cudaMemsetAsync(sigmabar, 0, sizeof(float) * KG, st))))
                return COV_ERR_CUDA;
        }
        const int Tm = T * m;
        for (int k = K; k >= 1; --k) {
            launch_pdl(back_scale_kernel, dim3((Tm + 255) / 256), dim3(256), 0, st, bb.ubar, prob->eta, Tm, bb.vbar);
            q = lqr_vjp_ws(ctx, rest, rest_bytes, n, m, sb.B, sb.gains, prob->Q, bb.vbar, T, bb.abb, st);
            if (q != COV_OK) return q;
            launch_pdl(narrow_kernel, dim3(nb), dim3(256), 0, st, bb.abb, T, n, d, bb.abf);
            launch_pdl(extract_kernel, dim3(nb), dim3(256), 0, st, hist + (size_t)(k - 1) * ss, T, n, d, sb.x);
            q = svgd_vjp_ws(ctx, rest, rest_bytes, sb.x, T, d, nullptr, &prob->gmm, prob->h, bb.abf, bb.xbar, nullptr,
                            wbar, mubar, sigmabar, k != K ? 1 : 0, st);
            if (q != COV_OK) return q;
            launch_pdl(lift_bar_kernel, dim3(nb), dim3(256), 0, st, bb.xbar, T, n, d, bb.sbar);
            q = rollout_vjp_ws(ctx, rest, rest_bytes, n, m, sb.A, sb.B, bb.sbar, T, bb.ub2, bb.lam0, st);
            if (q != COV_OK) return q;
            launch_pdl(back_accum_kernel, dim3((Tm + 255) / 256), dim3(256), 0, st, bb.ubar, bb.ub2, Tm, s0bar,
                       bb.lam0, n);
        }
        if (u0bar &&
            cuda_failed(ctx, cudaMemcpyAsync(u0bar, bb.ubar, sizeof(double) * Tm, cudaMemcpyDeviceToDevice, st)))
            return COV_ERR_CUDA;
        return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;
    };
    uint64_t key = 6700417ull;
    key = fnv(prob, sizeof(cov_problem), key);
    key = fnv(prob->gmm.w, sizeof(float) * KG, key);
    key = fnv(prob->gmm.mu, sizeof(float) * KG * d, key);
    key = fnv(prob->gmm.sigma, sizeof(float) * KG, key);
    key = fnv(&K, sizeof(K), key);
    key = fnv(&mode, sizeof(mode), key);
    const void* ptrs[10] = {u0, s_hist, sbar_K, wbar, mubar, sigmabar, s0bar, u0bar, ctx->ws,
                            reinterpret_cast<const void*>(ctx->ws_bytes)};
    key = fnv(ptrs, sizeof(ptrs), key);
    return run_cached_graph(ctx, ctx->back_graph, key, stream0, work);
}
