// cov_internal.h -- host-side internals of libcov: the context, the
// workspace bump allocator and launch helpers.  Not part of the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/cov.h"

struct cov_graph_cache {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    // identity of what was captured
    uint64_t key = 0;
};

#include <vector>

namespace cov {
struct SkTape;
}

struct cov_ctx {
    int device = 0;
    int num_sms = 148;
    void* ws = nullptr;        // workspace base
    size_t ws_bytes = 0;
    unsigned* status = nullptr;  // device status word (own allocation)
    // options
    int rows_per_thread = 4;
    int threads = 128;
    int ctas_per_sm = 8;
    int use_graph = 1;
    int use_tc = 2;            // tensor-core exponents: 0 off, 1 on, 2 for launches of >= 2^30 pairs
    int batch_share = 12;      // cov_solve_batched: percent of the GPU's CTA slots a problem's all-pairs launches plan for
    int plan_share = 100;      // the share the planner uses now (batch_share while a batch is enqueued)
    long long spin_limit = 1LL << 22;
    std::string last_cuda_error;
    cov_graph_cache solve_graph;
    cov_graph_cache batch_graph;       // cov_solve_batched: one outer iteration of all problems
    cov_graph_cache ckpt_graph;        // recording cov_solve_checkpointed: all its outer iterations
    cov_graph_cache back_graph;        // cov_solve_backward: the whole reverse sweep
    std::vector<cudaStream_t> pool;    // streams the batched graph's branches are captured on
    // cached LTI Riccati gains of cov_solve (valid while key matches; every
    // other call that writes workspace scratch clears the key)
    uint64_t gains_key = 0;
    // forward records of a taped cov_solve_checkpointed, one per outer
    // iteration, valid for cov_solve_backward while tape_key matches
    uint64_t tape_key = 0;
    // warm-started Sinkhorn potentials of cov_solve (valid while key matches)
    uint64_t pot_key = 0;
    std::vector<cov::SkTape> tapes;
};

namespace cov {

// Sequential 256-byte-aligned carving of the workspace.  `base == nullptr`
// only measures.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

inline size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

// Records a CUDA error on the context; returns true if `e` is an error.
bool cuda_failed(cov_ctx* ctx, cudaError_t e);

// Launch with programmatic stream serialisation allowed: the kernel may
// start while the previous grid in the stream finishes, and must begin with
// pdl_prologue() (cov_device.cuh) before touching global memory.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// A call is about to write scratch over the workspace: forget what cov_solve
// cached there (time-invariant gains, forward records).
inline void clobber_ws_caches(cov_ctx* ctx) {
    ctx->gains_key = 0;
    ctx->tape_key = 0;
    ctx->pot_key = 0;
}

// ---- per-component entry points used by cov_solve ---------------------------
// Workspace requirements of each component (bytes, 256-aligned pieces).
size_t sinkhorn_ws_bytes(int T, int M, int d);
size_t svgd_ws_bytes(int T, int d);
size_t lqr_ws_bytes(int T, int n, int m);

// Field calls on an explicit workspace region (cov_solve carves its own
// buffers first and passes the rest).
// scal_given: device [16] floats from sinkhorn_reference_stats (centre of y,
// 1/sum b), or nullptr to compute them in this call.
cov_status sinkhorn_field_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int x_ld, int T,
                             const float* y, const float* b, int M, int d, float eps, int n_iter, int flags,
                             float* f, float* g, float* p, float* a_out, cudaStream_t stream,
                             const float* scal_given = nullptr, float eps_start = 0.f, float eps_decay = 1.f);
// Forward record of a fixed-iteration, cold-start Sinkhorn run (device
// arrays inside the workspace), everything the adjoint needs.  Column terms
// are in the base-2 prescaled form of the forward kernels:
//   xhat = (x - centre) / sigma, sigma = sqrt(eps ln 2),
//   hx^t = log2 a + f^t/(eps ln 2) - |xhat|^2, hy^t = log2 b + g^t/(eps ln 2) - |yhat|^2,
//   hp^t = log2 a + p^t/(eps ln 2) - |xhat|^2;  padding entries hold -1e30.
struct SkTape {
    int n_iter, T, M, d, Tp, Mp;
    float eps, sigma, log2a;
    const float* xs;  // [d][Tp] xhat (padding 0)
    const float* ys;  // [d][Mp] yhat
    const float* lb;  // [Mp] log2 of the normalised weights
    const float* scal;  // [16]: centre of y, 1/sum b (0 for uniform weights)
    float* hx;        // [n+1][Tp]: slot t = hx^t (slot 0 the cold start; n = 0: the field's normaliser)
    float* hy;        // [n+1][Mp]: slot t = hy^t (slot 0 the cold start)
    float* hp;        // [n+2][Tp]: slot t = hp^t; slot n+1 = one more update (self-field normaliser)
    float* Df;        // [n+1][d][Tp]: slot t = sum_j pi^f_ij (yhat_j - xhat_i) of the f-update t
    float* Dg;        // [n+1][d][Mp]: slot t = sum_i pi^g_ji (xhat_i - yhat_j) of the g-update t
    float* Dp;        // [n+1][d][Tp]: slot t = sum_k pi^p_ik (xhat_k - xhat_i) of the p-update t
};
size_t sinkhorn_tape_bytes(int T, int M, int d, int n_iter, bool with_part = true);
// Bytes of the split buffers (partials and tickets) of a Sinkhorn run.
size_t sinkhorn_split_bytes(int T, int M, int d);
// Runs the recorded forward; *used = the workspace bytes it occupies (the
// tape must stay untouched while the adjoint reads it).  split_ws: the split
// buffers (sinkhorn_split_bytes) kept outside the tape, or nullptr to carve
// them inside it.  a_out [T][d]: the field of the recorded potentials, or
// nullptr.
cov_status sinkhorn_tape_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int x_ld, int T,
                            const float* y, const float* b, int M, int d, float eps, int n_iter,
                            const float* scal_given, SkTape* tape, size_t* used, cudaStream_t stream,
                            float* split_ws = nullptr, float* a_out = nullptr);
// Reverse mode of the field (adjoint.cu).  abar [T][abar_ld] FP32 device (the
// first d entries of each row are used), xbar [T][xbar_ld] written;
// ybar [M][d] and bbar [M] (NULL for uniform weights) written, or added to
// when accumulate != 0.
size_t sinkhorn_vjp_bytes(int T, int M, int d, int n_iter);
// given_tape: a forward record of exactly this x (then ws only holds the
// reverse sweep's buffers, sinkhorn_vjp_bytes_given), or nullptr to record
// one now at the start of ws.
size_t sinkhorn_vjp_bytes_given(int T, int M, int d);
cov_status sinkhorn_vjp_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int x_ld, int T,
                           const float* y, const float* b, int M, int d, float eps, int n_iter,
                           const float* scal_given, const float* abar, int abar_ld, float* xbar, int xbar_ld,
                           float* ybar, float* bbar, int accumulate, cudaStream_t stream,
                           const SkTape* given_tape = nullptr);
// Statistics of a reference set that every field evaluation on it needs:
// scal[0..d) = mean of y, scal[8] = 1 / sum b (0 when b == NULL).
void sinkhorn_reference_stats(const float* y, int M, int d, const float* b, float* scal, cudaStream_t stream);
// Score of a pixel-density reference at x [T][x_ld] (d = 2) into score [T][2].
cov_status density_score_launch(cov_ctx* ctx, const float* map, int H, int W, const float* x, int x_ld, int T,
                                float* score, cudaStream_t stream);
cov_status svgd_field_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int x_ld, int T, int d,
                         const float* score, const cov_gmm* gmm, float h, float* a_out, cudaStream_t stream);
// The Stein field of a short trajectory (T <= 1024) in one launch, reading
// the points as x[j x_ld + c] (FP64 states when x_double); COV_ERR_UNSUPPORTED
// for longer ones.  svgd_field_ws takes it itself where it applies.
cov_status svgd_field_small(cov_ctx* ctx, const void* x, bool x_double, int x_ld, int T, int d, const float* score,
                            const cov_gmm* gmm, float h, float* a_out, cudaStream_t stream);
// Reverse mode of the Stein field (svgd_vjp.cu) on an explicit workspace:
// x, abar [T][d] row-major; score [T][d] or nullptr (then the mixture's);
// xbar [T][d] written; sbar [T][d] or nullptr; the mixture gradients
// wbar [K], mubar [K][d], sigmabar [K] written (accumulate = 0) or added to.
size_t svgd_vjp_ws_bytes(int T, int d, int K, int num_sms);
cov_status svgd_vjp_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int T, int d, const float* score,
                       const cov_gmm* gmm, float h, const float* abar, float* xbar, float* sbar, float* wbar,
                       float* mubar, float* sigmabar, int accumulate, cudaStream_t st);
cov_status lqr_track_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const double* A, const double* B,
                        const double* Q, const double* R, const double* abar, int T, int n, int m,
                        double* v_out, double* z_out, cudaStream_t stream);

// Pair-tile scheduling of the all-pairs kernels.
struct SplitPlan {
    int n_rb;        // row blocks
    int splits;      // column splits
    int cols_per_split;  // multiple of the planning unit (8 columns; 256 for the tensor-core kernel)
};
// max_waves bounds the split count searched: at most about max_waves waves
// of CTAs over the slots.
SplitPlan plan_splits(int n_rows, int n_cols, int rows_per_cta, int slots, int unit = 8, int fixed = 64,
                      int max_waves = 2);

// A one-wave plan that uses exactly `budget` CTAs: every row block gets s or
// s + 1 column splits (the first n_hi row blocks s + 1), so that with budget
// = resident capacity every SM holds the same number of CTAs of nearly the
// same work.  (With a uniform split count the grid falls short of the
// capacity, and the SMs that hold a full complement finish last.)  Seg has
// the fields n_rb, splits, n_hi, cols_per_split, cps_lo.  With few splits
// per row block, s and s + 1 splits differ too much in work per CTA
// (measured slower for s = 1); with fewer than min_units planning units per
// split, rounding would leave whole CTAs without columns: the uniform plan
// is kept then.
template <class Seg>
inline void fill_plan(Seg& a, int n_cols, int budget, int unit, int min_units) {
    const int units = (n_cols + unit - 1) / unit;
    const long long total = (long long)budget < (long long)a.n_rb * units ? (long long)budget : (long long)a.n_rb * units;
    const int s = (int)(total / a.n_rb);
    const int extra = (int)(total - (long long)s * a.n_rb);
    if (s < 3 || units / (s + 1) < min_units) return;
    if (extra == 0) {
        a.splits = s;
        a.n_hi = a.n_rb;
        a.cols_per_split = (units + s - 1) / s * unit;
        a.cps_lo = a.cols_per_split;
    } else {
        a.splits = s + 1;
        a.n_hi = extra;
        a.cols_per_split = (units + s) / (s + 1) * unit;
        a.cps_lo = (units + s - 1) / s * unit;
    }
}

// GMM descriptor passed by value to kernels.
struct GmmParams {
    int K;
    int d;
    float lw[COV_MAX_GMM];          // log2 of normalised weight - d log2 sigma
    float inv2s2[COV_MAX_GMM];      // 1 / (2 sigma^2 ln 2)   (base-2 exponent scale)
    float invs2[COV_MAX_GMM];       // 1 / sigma^2
    float mu[COV_MAX_GMM * COV_MAX_D];
};
cov_status make_gmm_params(const cov_gmm* g, int d, GmmParams* out);

}  // namespace cov
