// svgd_vjp.cu -- reverse mode of the Stein variational field (Eq. 4) and of
// the Gaussian-mixture score it uses, on sm_103a.
//
// For L = <abar, g> with g_l = 1/T sum_j k_lj [ s_j + (x_l - x_j) / h^2 ],
// k_lj = exp(-|x_l - x_j|^2 / (2 h^2)), the product rule over both roles of a
// point (row l and column j = l) gives, with r = x_l - x_j, delta = abar_l -
// abar_j and psi = abar_l . s_j + abar_j . s_l + delta . r / h^2:
//   xbar_l = 1/(T h^2) sum_j k_lj [ delta - r psi ]      (score held fixed)
//   sbar_l = 1/T       sum_j k_lj abar_j                  (dL/ds_l)
// Both are one all-pairs pass over rows l and columns j.  In the scaled
// coordinates z = x / (h c), c = sqrt(2 ln 2), the kernel is k = 2^(-|z_l -
// z_j|^2) (one MUFU.EX2) and with sh = h s / c, dz = z_l - z_j:
//   psi_hat = abar_l . sh_j + abar_j . sh_l + delta . dz,
//   xbar_l = 1/(T h^2) [ abar_l S0 - A - 2 ln2 W ],
//   S0 = sum_j k, A = sum_j k abar_j, W = sum_j (k psi_hat) dz,
// 6d + 3 FP32 operations and one exponential per pair (18 at d = 2).
//
// The mixture score's own reverse mode (Hessian of log q applied to sbar,
// and the gradients with respect to the weights, means and standard
// deviations) runs per point after the pass; its per-CTA sums of the
// mixture gradients are added in CTA order (deterministic).
#include <math.h>

#include <algorithm>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace cov {
namespace {

constexpr int kVThreads = 128;  // rows per CTA (one per thread)
constexpr int kVTile = 128;     // columns staged in shared memory per tile
constexpr int kGThreads = 256;  // points per CTA of the mixture reverse pass

// Mixture as plain arrays (raw weights, means, standard deviations).
struct GmmRaw {
    int K;
    float w[COV_MAX_GMM];
    float sigma[COV_MAX_GMM];
    float mu[COV_MAX_GMM * COV_MAX_D];
};

struct VjpBufs {
    int Tp;
    float* cols;    // [3d][Tp]: z, sh, abar (SoA)
    float* score;   // [T][d] the mixture score at x (gmm input)
    float* sbar;    // [T][d] dL/dscore when the caller gives no buffer
    float* part;    // [1 + 2d][splits][Tp]: S0, A, W partials
    double* gpart;  // [n_gcta][K][d + 2]: per-CTA mixture gradients
};

// Score of the mixture at one point: softmax responsibilities of the
// component log terms (natural base, max-subtracted), sum r_k (mu_k - x) / sigma_k^2.
template <int D>
__device__ void mixture_score(const GmmRaw& G, const float* xv, float* sc) {
    float m = -INFINITY;
    for (int k = 0; k < G.K; ++k) {
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float t = xv[c] - G.mu[k * COV_MAX_D + c];
            d2 = fmaf(t, t, d2);
        }
        const float s2 = G.sigma[k] * G.sigma[k];
        m = fmaxf(m, logf(G.w[k]) - D * logf(G.sigma[k]) - 0.5f * d2 / s2);
    }
    float tot = 0.f, acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0.f;
    for (int k = 0; k < G.K; ++k) {
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float t = xv[c] - G.mu[k * COV_MAX_D + c];
            d2 = fmaf(t, t, d2);
        }
        const float s2 = G.sigma[k] * G.sigma[k];
        const float r = expf(logf(G.w[k]) - D * logf(G.sigma[k]) - 0.5f * d2 / s2 - m);
        tot += r;
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = fmaf(r / s2, G.mu[k * COV_MAX_D + c] - xv[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) sc[c] = acc[c] / tot;
}

// Columns in scaled form: z = x / (h c), sh = h s / c, abar; the mixture
// score first when no score is given.
template <int D>
__global__ void svgd_vjp_prep_kernel(const float* __restrict__ x, const float* __restrict__ score, GmmRaw G,
                                     int use_gmm, const float* __restrict__ abar, int T, int Tp, float zscale,
                                     float sscale, float* __restrict__ cols, float* __restrict__ score_out,
                                     unsigned* status) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    float xv[D], sv[D];
#pragma unroll
    for (int c = 0; c < D; ++c) xv[c] = x[(size_t)i * D + c];
    if (use_gmm) {
        mixture_score<D>(G, xv, sv);
#pragma unroll
        for (int c = 0; c < D; ++c) score_out[(size_t)i * D + c] = sv[c];
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) sv[c] = score[(size_t)i * D + c];
    }
    bool ok = true;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const float av = abar[(size_t)i * D + c];
        cols[(size_t)c * Tp + i] = xv[c] * zscale;
        cols[(size_t)(D + c) * Tp + i] = sv[c] * sscale;
        cols[(size_t)(2 * D + c) * Tp + i] = av;
        ok &= finitef(xv[c]) && finitef(sv[c]) && finitef(av);
    }
    if (!ok) raise_status(status, kDevNonfinite);
}

// The all-pairs pass: CTA (row block bx, column split by) accumulates, for
// its 128 rows, S0, A and W over the columns of its split; partials go to
// part[comp][split][row].  Column tiles are staged in shared memory, the
// next tile's values held in registers while the current one is consumed.
template <int D>
__global__ void __launch_bounds__(kVThreads) svgd_vjp_pairs_kernel(const float* __restrict__ cols, int T, int Tp,
                                                                   int cols_per_split, float* __restrict__ part) {
    pdl_prologue();
    constexpr int NC = 3 * D;
    __shared__ __align__(16) float st[NC][kVTile];
    const int tid = threadIdx.x;
    const int l = blockIdx.x * kVThreads + tid;
    const int split = blockIdx.y, splits = gridDim.y;
    const int c0 = split * cols_per_split;
    const int c1 = min(T, c0 + cols_per_split);
    float zl[D], sl[D], al[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const bool live = l < T;
        zl[c] = live ? cols[(size_t)c * Tp + l] : 0.f;
        sl[c] = live ? cols[(size_t)(D + c) * Tp + l] : 0.f;
        al[c] = live ? cols[(size_t)(2 * D + c) * Tp + l] : 0.f;
    }
    float S0 = 0.f, A[D], W[D];
#pragma unroll
    for (int c = 0; c < D; ++c) A[c] = W[c] = 0.f;
    // this thread's column of the next tile
    float nxt[NC];
    auto fetch = [&](int base) {
        const int j = base + tid;
#pragma unroll
        for (int k = 0; k < NC; ++k) nxt[k] = j < c1 ? cols[(size_t)k * Tp + j] : 0.f;
    };
    if (c0 < c1) fetch(c0);
    for (int base = c0; base < c1; base += kVTile) {
        __syncthreads();  // the previous tile is consumed
#pragma unroll
        for (int k = 0; k < NC; ++k) st[k][tid] = nxt[k];
        __syncthreads();
        if (base + kVTile < c1) fetch(base + kVTile);
        const int n = min(kVTile, c1 - base);
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            float dz[D], q = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                dz[c] = zl[c] - st[c][j];
                q = fmaf(dz[c], dz[c], q);
            }
            const float k = ex2(-q);
            float psi = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float aj = st[2 * D + c][j];
                psi = fmaf(al[c], st[D + c][j], psi);
                psi = fmaf(aj, sl[c], psi);
                psi = fmaf(al[c] - aj, dz[c], psi);
                A[c] = fmaf(k, aj, A[c]);
            }
            const float kp = k * psi;
            S0 += k;
#pragma unroll
            for (int c = 0; c < D; ++c) W[c] = fmaf(kp, dz[c], W[c]);
        }
    }
    if (l < T) {
        const size_t cs = (size_t)splits * Tp;
        float* P = part + (size_t)split * Tp + l;
        P[0] = S0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            P[(1 + c) * cs] = A[c];
            P[(1 + D + c) * cs] = W[c];
        }
    }
}

// Sum the splits in split order and form xbar and sbar (row-major [T][d]).
template <int D>
__global__ void svgd_vjp_reduce_kernel(const float* __restrict__ part, const float* __restrict__ cols, int T, int Tp,
                                       int splits, float inv_th2, float inv_t, float* __restrict__ xbar,
                                       float* __restrict__ sbar, unsigned* status) {
    pdl_prologue();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= T) return;
    const size_t cs = (size_t)splits * Tp;
    float S0 = 0.f, A[D], W[D];
#pragma unroll
    for (int c = 0; c < D; ++c) A[c] = W[c] = 0.f;
    for (int s = 0; s < splits; ++s) {
        const float* P = part + (size_t)s * Tp + l;
        S0 += P[0];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            A[c] += P[(1 + c) * cs];
            W[c] += P[(1 + D + c) * cs];
        }
    }
    bool ok = true;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const float al = cols[(size_t)(2 * D + c) * Tp + l];
        const float xb = inv_th2 * (al * S0 - A[c] - 2.0f * 0.69314718055994531f * W[c]);
        const float sb = inv_t * A[c];
        xbar[(size_t)l * D + c] = xb;
        sbar[(size_t)l * D + c] = sb;
        ok &= finitef(xb) && finitef(sb);
    }
    if (!ok) raise_status(status, kDevNonfinite);
}

// Sum of one value per thread over the CTA in a fixed order; the total is
// returned to thread 0.
__device__ double block_sum_d(double v, double* red) {
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

// Reverse mode of the mixture score per point, for c = sbar_i: with the
// responsibilities r_k, u_k = (mu_k - x) / sigma_k^2, S = sum_k r_k u_k and
// beta_k = r_k (c . u_k - c . S):
//   xbar_i  += sum_k [ beta_k u_k - r_k c / sigma_k^2 ]
//   mubar_k += -beta_k u_k + r_k c / sigma_k^2
//   sigmabar_k += beta_k (-d / sigma_k + |x - mu_k|^2 / sigma_k^3) - 2 r_k (c . u_k) / sigma_k
//   wbar_k  += beta_k / w_k
// The mixture sums of this CTA's points are written to gpart[cta][k][0..d+2)
// as (mubar (d), sigmabar, wbar).
template <int D>
__global__ void __launch_bounds__(kGThreads) gmm_vjp_kernel(const float* __restrict__ x, GmmRaw G,
                                                            const float* __restrict__ sbar, int T,
                                                            float* __restrict__ xbar, double* __restrict__ gpart) {
    pdl_prologue();
    __shared__ double red[kGThreads / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < T;
    float xv[D], cv[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        xv[c] = live ? x[(size_t)i * D + c] : 0.f;
        cv[c] = live ? sbar[(size_t)i * D + c] : 0.f;
    }
    // responsibilities: log terms, their maximum and normaliser
    float m = -INFINITY;
    for (int k = 0; k < G.K; ++k) {
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float t = xv[c] - G.mu[k * COV_MAX_D + c];
            d2 = fmaf(t, t, d2);
        }
        m = fmaxf(m, logf(G.w[k]) - D * logf(G.sigma[k]) - 0.5f * d2 / (G.sigma[k] * G.sigma[k]));
    }
    float tot = 0.f, S[D];
#pragma unroll
    for (int c = 0; c < D; ++c) S[c] = 0.f;
    for (int k = 0; k < G.K; ++k) {
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float t = xv[c] - G.mu[k * COV_MAX_D + c];
            d2 = fmaf(t, t, d2);
        }
        const float s2 = G.sigma[k] * G.sigma[k];
        const float r = expf(logf(G.w[k]) - D * logf(G.sigma[k]) - 0.5f * d2 / s2 - m);
        tot += r;
#pragma unroll
        for (int c = 0; c < D; ++c) S[c] = fmaf(r / s2, G.mu[k * COV_MAX_D + c] - xv[c], S[c]);
    }
    const float inv_tot = 1.f / tot;
    float cS = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        S[c] *= inv_tot;
        cS = fmaf(cv[c], S[c], cS);
    }
    float xb[D];
#pragma unroll
    for (int c = 0; c < D; ++c) xb[c] = 0.f;
    for (int k = 0; k < G.K; ++k) {
        float d2 = 0.f, u[D], cu = 0.f;
        const float s2 = G.sigma[k] * G.sigma[k];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float t = xv[c] - G.mu[k * COV_MAX_D + c];
            d2 = fmaf(t, t, d2);
            u[c] = -t / s2;
            cu = fmaf(cv[c], u[c], cu);
        }
        const float r = live ? expf(logf(G.w[k]) - D * logf(G.sigma[k]) - 0.5f * d2 / s2 - m) * inv_tot : 0.f;
        const float beta = r * (cu - cS);
        float mb[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xb[c] = fmaf(beta, u[c], xb[c]) - r * cv[c] / s2;
            mb[c] = -beta * u[c] + r * cv[c] / s2;
        }
        const float sb = beta * (-D / G.sigma[k] + d2 / (s2 * G.sigma[k])) - 2.f * r * cu / G.sigma[k];
        const float wb = beta / G.w[k];
        double* out = gpart + ((size_t)blockIdx.x * G.K + k) * (D + 2);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double t = block_sum_d(live ? (double)mb[c] : 0.0, red);
            if (threadIdx.x == 0) out[c] = t;
        }
        const double ts = block_sum_d(live ? (double)sb : 0.0, red);
        const double tw = block_sum_d(live ? (double)wb : 0.0, red);
        if (threadIdx.x == 0) {
            out[D] = ts;
            out[D + 1] = tw;
        }
    }
    if (live) {
#pragma unroll
        for (int c = 0; c < D; ++c) xbar[(size_t)i * D + c] += xb[c];
    }
}

// Mixture gradients: the per-CTA sums added in CTA order.
__global__ void gmm_vjp_sum_kernel(const double* __restrict__ gpart, int n_cta, int K, int d, float* __restrict__ wbar,
                                   float* __restrict__ mubar, float* __restrict__ sigmabar, int accumulate) {
    pdl_prologue();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (k, component)
    const int per = d + 2;
    if (e >= K * per) return;
    const int k = e / per, c = e % per;
    double s = 0.0;
    for (int b = 0; b < n_cta; ++b) s += gpart[((size_t)b * K + k) * per + c];
    float* out = c < d ? (mubar ? mubar + (size_t)k * d + c : nullptr) : (c == d ? (sigmabar ? sigmabar + k : nullptr)
                                                                             : (wbar ? wbar + k : nullptr));
    if (out) *out = accumulate ? *out + (float)s : (float)s;
}

int vjp_splits(int T, int num_sms) {
    const int n_rb = (T + kVThreads - 1) / kVThreads;
    const int tiles = (T + kVTile - 1) / kVTile;
    const int target = 8 * num_sms;  // CTAs of 128 threads: several per SM
    return std::max(1, std::min(tiles, target / n_rb));
}

VjpBufs carve_vjp(Carver& cv, int T, int d, int K, int splits, bool with_gmm) {
    VjpBufs B{};
    B.Tp = (int)round_up((size_t)T, 256);
    B.cols = cv.take<float>((size_t)3 * d * B.Tp);
    B.score = with_gmm ? cv.take<float>((size_t)T * d) : nullptr;
    B.sbar = cv.take<float>((size_t)T * d);
    B.part = cv.take<float>((size_t)(1 + 2 * d) * splits * B.Tp);
    const int n_gcta = (T + kGThreads - 1) / kGThreads;
    B.gpart = with_gmm ? cv.take<double>((size_t)n_gcta * K * (d + 2)) : nullptr;
    return B;
}

template <int D>
cov_status svgd_vjp_d(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int T, const float* score,
                      const GmmRaw* G, float h, const float* abar, float* xbar, float* sbar, float* wbar,
                      float* mubar, float* sigmabar, int accumulate, cudaStream_t st) {
    const bool use_gmm = score == nullptr;
    const int splits = vjp_splits(T, ctx->num_sms);
    Carver cv(ws);
    VjpBufs B = carve_vjp(cv, T, D, use_gmm ? G->K : 0, splits, use_gmm);
    if (!ws || cv.off > ws_bytes) return COV_ERR_WORKSPACE;
    const double c = sqrt(2.0 * 0.69314718055994531);
    GmmRaw Gv = use_gmm ? *G : GmmRaw{};
    float* sb = sbar ? sbar : B.sbar;
    const int nb = (T + 255) / 256;
    launch_pdl(svgd_vjp_prep_kernel<D>, dim3(nb), dim3(256), 0, st, x, score, Gv, use_gmm ? 1 : 0, abar, T, B.Tp,
               (float)(1.0 / (h * c)), (float)(h / c), B.cols, B.score, ctx->status);
    const int cps = (int)round_up((size_t)((T + splits - 1) / splits), kVTile);
    const int n_split = (T + cps - 1) / cps;
    launch_pdl(svgd_vjp_pairs_kernel<D>, dim3((T + kVThreads - 1) / kVThreads, n_split), dim3(kVThreads), 0, st,
               (const float*)B.cols, T, B.Tp, cps, B.part);
    launch_pdl(svgd_vjp_reduce_kernel<D>, dim3(nb), dim3(256), 0, st, (const float*)B.part, (const float*)B.cols, T,
               B.Tp, n_split, (float)(1.0 / ((double)T * h * h)), (float)(1.0 / T), xbar, sb, ctx->status);
    if (use_gmm) {
        const int n_gcta = (T + kGThreads - 1) / kGThreads;
        launch_pdl(gmm_vjp_kernel<D>, dim3(n_gcta), dim3(kGThreads), 0, st, x, Gv, (const float*)sb, T, xbar,
                   B.gpart);
        if (wbar || mubar || sigmabar) {
            const int ne = Gv.K * (D + 2);
            launch_pdl(gmm_vjp_sum_kernel, dim3((ne + 127) / 128), dim3(128), 0, st, (const double*)B.gpart, n_gcta,
                       Gv.K, D, wbar, mubar, sigmabar, accumulate);
        }
    }
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

}  // namespace

size_t svgd_vjp_ws_bytes(int T, int d, int K, int num_sms) {
    Carver cv(nullptr);
    carve_vjp(cv, T, d, K, vjp_splits(T, num_sms), true);
    return round_up(cv.off, 256);
}

// The mixture as plain arrays; COV_ERR_INVALID_ARG for an invalid descriptor.
static cov_status gmm_raw(const cov_gmm* gmm, int d, GmmRaw* G) {
    if (!gmm || gmm->K < 1 || gmm->K > COV_MAX_GMM || gmm->d != d || !gmm->w || !gmm->mu || !gmm->sigma)
        return COV_ERR_INVALID_ARG;
    *G = GmmRaw{};
    G->K = gmm->K;
    for (int k = 0; k < gmm->K; ++k) {
        if (!(gmm->w[k] > 0.f) || !(gmm->sigma[k] > 0.f) || !isfinite(gmm->w[k]) || !isfinite(gmm->sigma[k]))
            return COV_ERR_INVALID_ARG;
        G->w[k] = gmm->w[k];
        G->sigma[k] = gmm->sigma[k];
        for (int c = 0; c < d; ++c) {
            if (!isfinite(gmm->mu[k * d + c])) return COV_ERR_INVALID_ARG;
            G->mu[k * COV_MAX_D + c] = gmm->mu[k * d + c];
        }
    }
    return COV_OK;
}

cov_status svgd_vjp_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int T, int d, const float* score,
                       const cov_gmm* gmm, float h, const float* abar, float* xbar, float* sbar, float* wbar,
                       float* mubar, float* sigmabar, int accumulate, cudaStream_t st) {
    if (!ctx || !x || !abar || !xbar || T < 1 || d < 1 || d > COV_MAX_D || !(h > 0.f) || !isfinite(h))
        return COV_ERR_INVALID_ARG;
    GmmRaw G{};
    if (!score) {
        const cov_status r = gmm_raw(gmm, d, &G);
        if (r != COV_OK) return r;
    }
    const GmmRaw* gp = score ? nullptr : &G;
    switch (d) {
        case 1: return svgd_vjp_d<1>(ctx, ws, ws_bytes, x, T, score, gp, h, abar, xbar, sbar, wbar, mubar, sigmabar, accumulate, st);
        case 2: return svgd_vjp_d<2>(ctx, ws, ws_bytes, x, T, score, gp, h, abar, xbar, sbar, wbar, mubar, sigmabar, accumulate, st);
        case 3: return svgd_vjp_d<3>(ctx, ws, ws_bytes, x, T, score, gp, h, abar, xbar, sbar, wbar, mubar, sigmabar, accumulate, st);
        case 4: return svgd_vjp_d<4>(ctx, ws, ws_bytes, x, T, score, gp, h, abar, xbar, sbar, wbar, mubar, sigmabar, accumulate, st);
        case 5: return svgd_vjp_d<5>(ctx, ws, ws_bytes, x, T, score, gp, h, abar, xbar, sbar, wbar, mubar, sigmabar, accumulate, st);
        default: return svgd_vjp_d<6>(ctx, ws, ws_bytes, x, T, score, gp, h, abar, xbar, sbar, wbar, mubar, sigmabar, accumulate, st);
    }
}

}  // namespace cov

extern "C" size_t cov_workspace_size_svgd_vjp(int T, int d, int K) {
    if (T < 1 || d < 1 || d > COV_MAX_D || K < 0 || K > COV_MAX_GMM) return 0;
    // split count planned for up to 1024 SMs (the plan never needs more)
    return cov::svgd_vjp_ws_bytes(T, d, K, 1024) + 4096;
}

extern "C" cov_status cov_field_svgd_vjp(cov_ctx* ctx, const float* x, int T, int d, const float* score,
                                         const cov_gmm* gmm, float h, const float* abar, float* xbar, float* sbar,
                                         float* wbar, float* mubar, float* sigmabar, cov_stream_t stream) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::clobber_ws_caches(ctx);
    return cov::svgd_vjp_ws(ctx, ctx->ws, ctx->ws_bytes, x, T, d, score, gmm, h, abar, xbar, sbar, wbar, mubar,
                            sigmabar, 0, (cudaStream_t)stream);
}
