// ctx.cu -- context, workspace, status word and options of libcov.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "cov_device.cuh"
#include "cov_internal.h"

bool cov::cuda_failed(cov_ctx* ctx, cudaError_t e) {
    if (e == cudaSuccess) return false;
    if (ctx) ctx->last_cuda_error = cudaGetErrorString(e);
    return true;
}

namespace cov {
size_t solve_buffers_bytes(int T, int d, int n, int m, int M);
void drop_solve_graph(cov_ctx* ctx);
void destroy_stream_pool(cov_ctx* ctx);
void lqr_set_attributes();
}  // namespace cov

extern "C" const char* cov_status_string(cov_status s) {
    switch (s) {
        case COV_OK: return "COV_OK";
        case COV_ERR_INVALID_ARG: return "COV_ERR_INVALID_ARG";
        case COV_ERR_WORKSPACE: return "COV_ERR_WORKSPACE";
        case COV_ERR_CUDA: return "COV_ERR_CUDA";
        case COV_ERR_NONFINITE: return "COV_ERR_NONFINITE";
        case COV_ERR_TIMEOUT: return "COV_ERR_TIMEOUT";
        case COV_ERR_UNSUPPORTED: return "COV_ERR_UNSUPPORTED";
    }
    return "COV_ERR_UNKNOWN";
}

extern "C" cov_status cov_ctx_create(cov_ctx** out, int device, size_t workspace_bytes) {
    if (!out) return COV_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return COV_ERR_CUDA;
    cov_ctx* ctx = new (std::nothrow) cov_ctx();
    if (!ctx) return COV_ERR_WORKSPACE;
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cov::lqr_set_attributes();
    if (cudaMalloc(&ctx->status, 256) != cudaSuccess) {
        delete ctx;
        return COV_ERR_WORKSPACE;
    }
    if (cudaMemset(ctx->status, 0, 256) != cudaSuccess) {
        cudaFree(ctx->status);
        delete ctx;
        return COV_ERR_CUDA;
    }
    if (workspace_bytes) {
        if (cudaMalloc(&ctx->ws, workspace_bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(ctx->status);
            delete ctx;
            return COV_ERR_WORKSPACE;
        }
        ctx->ws_bytes = workspace_bytes;
    }
    *out = ctx;
    return COV_OK;
}

extern "C" void cov_ctx_destroy(cov_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    cov::drop_solve_graph(ctx);
    cov::destroy_stream_pool(ctx);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->status) cudaFree(ctx->status);
    delete ctx;
}

extern "C" cov_status cov_ctx_reserve(cov_ctx* ctx, size_t bytes) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    if (bytes <= ctx->ws_bytes) return COV_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    if (cov::cuda_failed(ctx, cudaDeviceSynchronize())) return COV_ERR_CUDA;
    cov::drop_solve_graph(ctx);
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cov::cuda_failed(ctx, cudaGetLastError());
        return COV_ERR_WORKSPACE;
    }
    ctx->ws = p;
    ctx->ws_bytes = bytes;
    return COV_OK;
}

extern "C" size_t cov_workspace_size(int T, int M, int d, int n, int m) {
    if (T < 1 || d < 1 || d > COV_MAX_D) return 0;
    size_t field = cov::svgd_ws_bytes(T, d);
    if (M > 0) field = std::max(field, cov::sinkhorn_ws_bytes(T, M, d));
    size_t lqr = 0, solve = 0;
    if (n > 0 && m > 0) {
        lqr = cov::lqr_ws_bytes(T, n, m);
        solve = cov::solve_buffers_bytes(T, d, n, m, M);
    }
    return solve + std::max(field, lqr) + 4096;
}

extern "C" cov_status cov_ctx_reserve_for(cov_ctx* ctx, int T, int M, int d, int n, int m) {
    const size_t b = cov_workspace_size(T, M, d, n, m);
    if (!b) return COV_ERR_INVALID_ARG;
    return cov_ctx_reserve(ctx, b);
}

extern "C" cov_status cov_get_device_status(cov_ctx* ctx, cov_stream_t stream, int* flags) {
    if (!ctx || !flags) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    if (cov::cuda_failed(ctx, cudaStreamSynchronize((cudaStream_t)stream))) return COV_ERR_CUDA;
    unsigned v = 0;
    if (cov::cuda_failed(ctx, cudaMemcpy(&v, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost)))
        return COV_ERR_CUDA;
    if (cov::cuda_failed(ctx, cudaMemset(ctx->status, 0, sizeof(unsigned)))) return COV_ERR_CUDA;
    *flags = (int)v;
    if (v & cov::kDevTimeout) return COV_ERR_TIMEOUT;
    if (v & (cov::kDevNonfinite | cov::kDevNotSpd)) return COV_ERR_NONFINITE;
    return COV_OK;
}

extern "C" const char* cov_last_cuda_error(cov_ctx* ctx) { return ctx ? ctx->last_cuda_error.c_str() : ""; }

extern "C" cov_status cov_ctx_set_option(cov_ctx* ctx, int key, long long value) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    switch (key) {
        case COV_OPT_ROWS_PER_THREAD:
            if (value != 2 && value != 4 && value != 8) return COV_ERR_INVALID_ARG;
            ctx->rows_per_thread = (int)value;
            break;
        case COV_OPT_THREADS:
            if (value != 128) return COV_ERR_INVALID_ARG;
            ctx->threads = (int)value;
            break;
        case COV_OPT_CTAS_PER_SM:
            if (value < 1 || value > 8) return COV_ERR_INVALID_ARG;
            ctx->ctas_per_sm = (int)value;
            break;
        case COV_OPT_USE_GRAPH:
            if (value != 0 && value != 1) return COV_ERR_INVALID_ARG;
            ctx->use_graph = (int)value;
            break;
        case COV_OPT_SPIN_LIMIT:
            if (value < 0) return COV_ERR_INVALID_ARG;
            ctx->spin_limit = value;
            break;
        case COV_OPT_TENSOR_CORES:
            if (value < 0 || value > 2) return COV_ERR_INVALID_ARG;
            ctx->use_tc = (int)value;
            break;
        case COV_OPT_BATCH_SHARE:
            if (value < 1 || value > 100) return COV_ERR_INVALID_ARG;
            ctx->batch_share = (int)value;
            if (ctx->batch_graph.exec) cudaGraphExecDestroy(ctx->batch_graph.exec);
            if (ctx->batch_graph.graph) cudaGraphDestroy(ctx->batch_graph.graph);
            ctx->batch_graph = cov_graph_cache{};
            break;
        default:
            return COV_ERR_INVALID_ARG;
    }
    cov::drop_solve_graph(ctx);
    return COV_OK;
}
