// autotune.cu -- tile-shape sweep of the all-pairs kernels through the
// library's own calls: rows per lane R and the resident-CTA cap are timed
// on the caller's inputs with CUDA events on the caller's stream, as the
// per-iteration cost (t(2 + n iterations) - t(2 iterations)) / n (n = 20
// below 2^30 pairs per iteration, 4 above) so that the prep and gradient
// launches cancel, and the fastest pair is applied to the context.
#include <math.h>

#include <algorithm>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace {

struct Candidate {
    int R, cps;
};
constexpr Candidate kCandidates[] = {{2, 8}, {4, 8}, {8, 8}, {4, 6}, {2, 6}, {8, 4}};
constexpr int kNumCandidates = sizeof(kCandidates) / sizeof(kCandidates[0]);

}  // namespace

extern "C" cov_status cov_autotune_sinkhorn(cov_ctx* ctx, const float* x, int T, const float* y, const float* b,
                                            int M, int d, float eps, int* best_R, int* best_ctas_per_sm,
                                            double* sweep, cov_stream_t stream) {
    if (!ctx || !x || !y || T < 1 || M < 1 || d < 1 || d > COV_MAX_D || !(eps > 0.f)) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int R0 = ctx->rows_per_thread, c0 = ctx->ctas_per_sm;
    // the shapes are those of the CUDA-core kernel: sweep that path whatever
    // the exponent setting (the tensor-core kernel has a single shape)
    const int tc0 = ctx->use_tc;
    cudaEvent_t e0, e1;
    if (cov::cuda_failed(ctx, cudaEventCreate(&e0))) return COV_ERR_CUDA;
    if (cov::cuda_failed(ctx, cudaEventCreate(&e1))) {
        cudaEventDestroy(e0);
        return COV_ERR_CUDA;
    }
    ctx->use_tc = 0;  // restored below on every path from here
    cov::clobber_ws_caches(ctx);
    cov_status r = COV_OK;
    double best = 1e300;
    int bR = R0, bC = c0;
    auto run = [&](int n) {
        return cov::sinkhorn_field_ws(ctx, ctx->ws, ctx->ws_bytes, x, d, T, y, b, M, d, eps, n, 0, nullptr, nullptr,
                                      nullptr, nullptr, st);
    };
    auto timed = [&](int n, float* ms) -> cov_status {
        if (cov::cuda_failed(ctx, cudaEventRecord(e0, st))) return COV_ERR_CUDA;
        const cov_status q = run(n);
        if (q != COV_OK) return q;
        if (cov::cuda_failed(ctx, cudaEventRecord(e1, st)) || cov::cuda_failed(ctx, cudaEventSynchronize(e1)) ||
            cov::cuda_failed(ctx, cudaEventElapsedTime(ms, e0, e1)))
            return COV_ERR_CUDA;
        return COV_OK;
    };
    // iterations timed per candidate: enough that the difference spans a few
    // hundred microseconds at small sizes (4 at the large ones)
    const double pairs_iter = 2.0 * T * (double)M + (double)T * T;
    const int n_diff = pairs_iter < (double)(1LL << 30) ? 20 : 4;
    for (int k = 0; k < kNumCandidates && r == COV_OK; ++k) {
        const Candidate c = kCandidates[k];
        ctx->rows_per_thread = c.R;  // the planner maps R to the built shapes for this d
        ctx->ctas_per_sm = c.cps;
        r = run(1);
        float lo[3], hi[3];
        for (int rep = 0; rep < 3 && r == COV_OK; ++rep) {
            r = timed(2, &lo[rep]);
            if (r == COV_OK) r = timed(2 + n_diff, &hi[rep]);
        }
        if (r != COV_OK) break;
        std::sort(lo, lo + 3);
        std::sort(hi, hi + 3);
        const double us = 1e3 * (hi[1] - lo[1]) / n_diff;
        if (sweep) {
            sweep[3 * k] = c.R;
            sweep[3 * k + 1] = c.cps;
            sweep[3 * k + 2] = us;
        }
        if (us < best) {
            best = us;
            bR = c.R;
            bC = c.cps;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->use_tc = tc0;
    if (r != COV_OK) {
        ctx->rows_per_thread = R0;
        ctx->ctas_per_sm = c0;
        return r;
    }
    cov_ctx_set_option(ctx, COV_OPT_ROWS_PER_THREAD, bR);  // also drops graphs planned with other shapes
    cov_ctx_set_option(ctx, COV_OPT_CTAS_PER_SM, bC);
    if (best_R) *best_R = bR;
    if (best_ctas_per_sm) *best_ctas_per_sm = bC;
    return COV_OK;
}
