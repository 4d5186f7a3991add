// peaks.cu -- issue-rate probes that give the roofline denominators of the
// all-pairs kernels on the running GPU: FP32 FMA, packed FP32x2 FMA, MUFU
// ex2 and FP64 FMA throughput, FP64 FMA latency and the SM clock; and the
// throughput and accuracy of 2^x on the FMA pipe (exp2_fma2).
#include <math.h>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace cov {

constexpr int kChains = 8;

__global__ void probe_ffma(int iters, float a, float b, float* out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.f) out[0] = s;
}

__global__ void probe_ffma2(int iters, float a, float b, float* out) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(threadIdx.x + c, c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma2(x[c], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == 12345.f) out[0] = s;
}

__global__ void probe_ex2(int iters, float* out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -(float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = ex2(x[c]);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.f) out[0] = s;
}

// 2^x on the FMA pipe (exp2_fma2), two values per call, same chain shape
__global__ void probe_exp2_fma(int iters, float* out) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(-(float)(threadIdx.x + c) * 1e-3f, -(float)c * 1e-2f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = exp2_fma2(x[c]);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == 12345.f) out[0] = s;
}

// Largest relative error of exp2_fma2 against FP64 exp2 on n points of
// [-125, 127]; written as the bit pattern of a non-negative float, which
// orders like the unsigned integer.
__global__ void probe_exp2_fma_error(int n, unsigned* max_bits) {
    unsigned worst = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; 2 * k + 1 < n; k += gridDim.x * blockDim.x) {
        const float x0 = -125.f + 252.f * (float)(2 * k) / (float)n;
        const float x1 = -125.f + 252.f * (float)(2 * k + 1) / (float)n;
        const float2 r = exp2_fma2(make_float2(x0, x1));
        const float e0 = (float)fabs((double)r.x / exp2((double)x0) - 1.0);
        const float e1 = (float)fabs((double)r.y / exp2((double)x1) - 1.0);
        worst = max(worst, max(__float_as_uint(e0), __float_as_uint(e1)));
    }
    atomicMax(max_bits, worst);
}

__global__ void probe_dfma(int iters, double a, double b, float* out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.0) out[0] = (float)s;
}

// One thread: dependent DFMA chain, cycles per FMA; and clock/globaltimer.
__global__ void probe_dfma_latency(int iters, double a, double b, float* out) {
    double x = threadIdx.x;
    const long long c0 = clock64();
    unsigned long long g0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
    for (int i = 0; i < iters; ++i) x = fma(x, a, b);
    const long long c1 = clock64();
    unsigned long long g1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
    if (threadIdx.x == 0) {
        out[1] = (float)((double)(c1 - c0) / iters);
        out[2] = (float)((double)(c1 - c0) / (double)(g1 - g0) * 1000.0);  // MHz
    }
    if (x == 12345.0) out[0] = (float)x;
}

}  // namespace cov

extern "C" cov_status cov_probe_peaks(cov_ctx* ctx, int iters, double* out, cov_stream_t stream) {
    using namespace cov;
    if (!ctx || !out || iters < 1) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    float* dev = nullptr;
    // the probe result slot lives in the status allocation (bytes 16..63)
    dev = reinterpret_cast<float*>(reinterpret_cast<char*>(ctx->status) + 16);
    cudaEvent_t e0, e1;
    if (cuda_failed(ctx, cudaEventCreate(&e0)) || cuda_failed(ctx, cudaEventCreate(&e1))) return COV_ERR_CUDA;
    const int blocks = ctx->num_sms * 8, threads = 256;
    const double lanes = (double)blocks * threads;
    float ms = 0.f;
    // warm-up
    probe_ffma<<<blocks, threads, 0, st>>>(iters / 4 + 1, 0.999f, 0.001f, dev);
    auto timed = [&](auto launch) -> double {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        return ms * 1e-3;
    };
    double t = timed([&] { probe_ffma<<<blocks, threads, 0, st>>>(iters, 0.999f, 0.001f, dev); });
    out[0] = lanes * kChains * iters / t;
    t = timed([&] { probe_ffma2<<<blocks, threads, 0, st>>>(iters, 0.999f, 0.001f, dev); });
    out[1] = 2.0 * lanes * kChains * iters / t;
    t = timed([&] { probe_ex2<<<blocks, threads, 0, st>>>(iters, dev); });
    out[2] = lanes * kChains * iters / t;
    const int diters = std::max(1, iters / 16);
    t = timed([&] { probe_dfma<<<blocks, threads, 0, st>>>(diters, 0.999, 0.001, dev); });
    out[3] = lanes * kChains * diters / t;
    t = timed([&] { probe_exp2_fma<<<blocks, threads, 0, st>>>(iters, dev); });
    out[6] = 2.0 * lanes * kChains * iters / t;
    probe_dfma_latency<<<1, 1, 0, st>>>(diters, 0.999, 0.001, dev);
    unsigned* err_bits = reinterpret_cast<unsigned*>(dev + 3);
    cudaMemsetAsync(err_bits, 0, sizeof(unsigned), st);
    probe_exp2_fma_error<<<ctx->num_sms * 4, 256, 0, st>>>(1 << 22, err_bits);
    float hv[4];
    cudaMemcpyAsync(hv, dev, sizeof(hv), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    out[4] = hv[1];
    out[5] = hv[2];
    out[7] = hv[3];  // the error bits read back as the float they are
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}
