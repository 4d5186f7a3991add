// divergence.cu -- value and gradient of the debiased Sinkhorn divergence of
// Eq. 6 at n_iter fixed log-domain iterations (the coverage loss of the
// differentiation workload), on sm_103a.
//
//   S = OT(p_s, q) - OT(p_s, p_s)/2 - OT(q, q)/2
//     = <a, f> + <b, g> - <a, p> - <b, q_self>
// with f, g the cross potentials and p the self potential of the trajectory
// samples after n_iter cold-start iterations (cov_field_sinkhorn), and q_self
// the self potential of the reference after as many iterations of the same
// averaged self update.  Each OT term is its dual value (after the last
// f-update the entropic correction of the cross term vanishes, and a
// symmetric problem's dual value is twice <a, p>).  Its gradient with
// respect to x_i is the envelope formula a_i times the descent field of
// Eq. 7 with the sign flipped: dS/dx_i = -(1/T) field_i.
#include <math.h>

#include <algorithm>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace cov {
namespace {

constexpr int kDivThreads = 1024;

struct DivBufs {
    float* f;  // [T]
    float* g;  // [M]
    float* p;  // [T]
    float* q;  // [M] (reference self potential, when computed here)
    float* a;  // [T][d] field
};

DivBufs carve_div(Carver& cv, int T, int M, int d, bool with_q) {
    DivBufs B{};
    B.f = cv.take<float>(T);
    B.g = cv.take<float>(M);
    B.p = cv.take<float>(T);
    B.q = with_q ? cv.take<float>(M) : nullptr;
    B.a = cv.take<float>((size_t)T * d);
    return B;
}

// Sum of one FP64 value per thread over the CTA, in a fixed order (warp
// shuffles, then the warp totals in warp order): deterministic.
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

// One CTA: value = sum f / T + sum bh g - sum p / T - sum bh q (bh = b /
// sum b, or 1/M), each sum in FP64 over fixed per-thread strides; and
// grad = -(1/T) a over the T x d field.
__global__ void div_value_kernel(const float* __restrict__ f, const float* __restrict__ g,
                                 const float* __restrict__ p, const float* __restrict__ q,
                                 const float* __restrict__ b, int T, int M, const float* __restrict__ a, int nd,
                                 double* __restrict__ value, float* __restrict__ grad, unsigned* status) {
    pdl_prologue();
    __shared__ double red[kDivThreads / 32];
    double sb = 0.0;
    if (b) {
        for (int j = threadIdx.x; j < M; j += blockDim.x) sb += (double)b[j];
        sb = block_sum(sb, red);
    }
    __shared__ double s_bsum;
    if (threadIdx.x == 0) s_bsum = b ? sb : (double)M;
    __syncthreads();
    const double inv_b = 1.0 / s_bsum;
    double sx = 0.0, sy = 0.0;
    for (int i = threadIdx.x; i < T; i += blockDim.x) sx += (double)f[i] - (double)p[i];
    for (int j = threadIdx.x; j < M; j += blockDim.x)
        sy += (b ? (double)b[j] : 1.0) * ((double)g[j] - (double)q[j]);
    sx = block_sum(sx, red);
    sy = block_sum(sy, red);
    if (threadIdx.x == 0) {
        const double v = sx / (double)T + sy * inv_b;
        *value = v;
        if (!isfinite(v)) raise_status(status, kDevNonfinite);
    }
    if (grad) {
        const float s = -1.0f / (float)T;
        for (int e = threadIdx.x; e < nd; e += blockDim.x) grad[e] = s * a[e];
    }
}

}  // namespace

size_t divergence_ws_bytes(int T, int M, int d) {
    Carver cv(nullptr);
    carve_div(cv, T, M, d, true);
    const size_t head = round_up(cv.off, 256);
    return head + std::max(sinkhorn_ws_bytes(T, M, d), sinkhorn_ws_bytes(M, M, d));
}

}  // namespace cov

extern "C" size_t cov_workspace_size_divergence(int T, int M, int d) {
    if (T < 1 || M < 1 || d < 1 || d > COV_MAX_D) return 0;
    return cov::divergence_ws_bytes(T, M, d) + 4096;
}

extern "C" cov_status cov_sinkhorn_divergence(cov_ctx* ctx, const float* x, int T, const float* y, const float* b,
                                              int M, int d, float eps, int n_iter, float* q_ref, int q_given,
                                              double* value, float* grad, cov_stream_t stream) {
    if (!ctx || !x || !y || !value || T < 1 || M < 1 || d < 1 || d > COV_MAX_D || n_iter < 0 || !(eps > 0.f) ||
        !isfinite(eps) || (q_given && !q_ref))
        return COV_ERR_INVALID_ARG;
    // the self potential of a weighted reference needs the weights inside
    // the self update, which the field kernels take as uniform
    if (!q_given && b) return COV_ERR_UNSUPPORTED;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::clobber_ws_caches(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    cov::Carver cv(ctx->ws);
    cov::DivBufs B = cov::carve_div(cv, T, M, d, !q_given && !q_ref);
    const size_t head = cov::round_up(cv.off, 256);
    if (!ctx->ws || head > ctx->ws_bytes) return COV_ERR_WORKSPACE;
    char* rest = static_cast<char*>(ctx->ws) + head;
    const size_t rest_bytes = ctx->ws_bytes - head;
    const float* q = q_given ? q_ref : (q_ref ? q_ref : B.q);
    if (!q_given) {
        // OT(q, q): the self potential of the reference, n_iter averaged self
        // updates over y (the p output of a field evaluation of y against itself)
        cov_status r = cov::sinkhorn_field_ws(ctx, rest, rest_bytes, y, d, M, y, nullptr, M, d, eps, n_iter, 0,
                                              nullptr, nullptr, const_cast<float*>(q), nullptr, st);
        if (r != COV_OK) return r;
    }
    // OT(p_s, q) and OT(p_s, p_s): cross potentials f, g, the trajectory's
    // self potential p and (for the gradient) the field
    cov_status r = cov::sinkhorn_field_ws(ctx, rest, rest_bytes, x, d, T, y, b, M, d, eps, n_iter, 0, B.f, B.g, B.p,
                                          grad ? B.a : nullptr, st);
    if (r != COV_OK) return r;
    cov::launch_pdl(cov::div_value_kernel, dim3(1), dim3(cov::kDivThreads), 0, st, B.f, B.g, B.p, q, b, T, M, B.a,
                    grad ? T * d : 0, value, grad, ctx->status);
    if (cov::cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}
