// noalloc.cu -- cov_field_sinkhorn_noalloc: the Sinkhorn-divergence field
// for callers that must not allocate device memory.
//
// Some host programs cannot call cudaMalloc: plugins whose host application
// owns every device byte and hands it out from its own arena, or real-time
// loops that cannot afford the implicit device-wide synchronisation of
// cudaMalloc/cudaFree.  For them this entry point takes its scratch (status
// word, prescaled points, column terms, tensor-core records, split partials
// and merge counters) from one fixed array compiled into the library instead
// of a context workspace.  The array costs kNoAllocBytes (48 MiB) on every
// GPU that loads the library, for the life of the process; a call needs at
// most sinkhorn_ws_bytes(T, M, d) of it, which for T = 65536 and
// M = 262144 is 35.4 / 41.1 / 46.9 / 35.6 / 41.4 / 47.1 MiB at d = 1..6.
#include <mutex>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(48) << 20;  // 48 MiB
constexpr size_t kStatusBytes = 256;                // status word + padding
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (the host-side symbol is only a stand-in, never a device address).
cov_status scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return COV_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return COV_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return COV_OK;
}

}  // namespace

extern "C" cov_status cov_field_sinkhorn_noalloc(const float* x, int T, const float* y, const float* b, int M, int d,
                                                 float eps, int n_iter, int flags, float* f, float* g, float* p,
                                                 float* a_out, cov_stream_t stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return COV_ERR_CUDA;
    }
    void* base = nullptr;
    const cov_status s = scratch_address(dev, &base);
    if (s != COV_OK) return s;
    // A host-side context describing the fixed array; it owns nothing.
    cov_ctx ctx;
    ctx.device = dev;
    if (cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return COV_ERR_CUDA;
    }
    ctx.status = static_cast<unsigned*>(base);
    char* ws = static_cast<char*>(base) + kStatusBytes;
    // Sizes whose scratch does not fit are rejected (COV_ERR_WORKSPACE)
    // before anything is launched; the merge counters are cleared on the
    // stream at the start of every call.
    return cov::sinkhorn_field_ws(&ctx, ws, kNoAllocBytes - kStatusBytes, x, d, T, y, b, M, d, eps, n_iter, flags,
                                  f, g, p, a_out, (cudaStream_t)stream);
}
