// cov_device.cuh -- sm_103a device helpers shared by the libcov kernels:
// inline-PTX wrappers for the special-function unit (ex2.approx), packed
// FP32x2 arithmetic, mbarriers and the bulk-copy (TMA) engine, plus the
// device status word.  Internal header of libcov; not part of the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cov {

// Status bits (mirrors COV_DEV_* of cov.h).
constexpr unsigned kDevNonfinite = 1u;
constexpr unsigned kDevTimeout = 2u;
constexpr unsigned kDevNotSpd = 4u;

// Column padding value of the log-domain kernels: exponent terms of padded
// columns are ~-1e30 and vanish after the running-max subtraction.
constexpr float kPadH = -1.0e30f;
// Initial running maximum (below any padded or real exponent).
constexpr float kNegBig = -3.0e38f;

__device__ __forceinline__ void raise_status(unsigned* st, unsigned bits) {
    if (st) atomicOr(st, bits);
}

// 2^x on the special-function unit (MUFU.EX2), flush-to-zero.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- packed FP32x2 arithmetic (one instruction, two lanes of work) -------
// (exp2_fma2, 2^x on the FMA pipe, follows the packed helpers below)
__device__ __forceinline__ uint64_t pk(float2 a) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 upk(uint64_t r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
// 2^x for two values on the FMA pipe (no MUFU): Cody–Waite range reduction,
// x = n + f with n = round(x) found by adding and subtracting 1.5 * 2^23
// (the sum's low mantissa bits then hold n) and f in [-1/2, 1/2]; 2^f by a
// degree-5 polynomial whose coefficients interpolate 2^f at the six
// Chebyshev nodes of [-1/2, 1/2] (max relative error 1.0e-7 with exact
// coefficients, 2.4e-7 evaluated in FP32, about that of ex2.approx); 2^n
// added to the exponent field as an integer.  x is clamped to [-125, 127]:
// below, the result is 2^-125 instead of a smaller number (negligible in
// the sums it feeds); above, 2^127 (finite but past any overflow guard).
__device__ __forceinline__ float2 exp2_fma2(float2 x) {
    x.x = fminf(fmaxf(x.x, -125.f), 127.f);
    x.y = fminf(fmaxf(x.y, -125.f), 127.f);
    const float2 shift = make_float2(12582912.f, 12582912.f);
    const float2 t = add2(x, shift);
    const float2 f = sub2(x, sub2(t, shift));
    float2 p = fma2(make_float2(1.3390863e-3f, 1.3390863e-3f), f, make_float2(9.6760318e-3f, 9.6760318e-3f));
    p = fma2(p, f, make_float2(5.5503570e-2f, 5.5503570e-2f));
    p = fma2(p, f, make_float2(2.4022107e-1f, 2.4022107e-1f));
    p = fma2(p, f, make_float2(6.9314718e-1f, 6.9314718e-1f));
    p = fma2(p, f, make_float2(1.0000001f, 1.0000001f));
    return make_float2(__int_as_float(__float_as_int(p.x) + (__float_as_int(t.x) << 23)),
                       __int_as_float(__float_as_int(p.y) + (__float_as_int(t.y) << 23)));
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// ---- mbarrier + bulk copy (cp.async.bulk, the TMA engine's 1-D path) ------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity; gives up after `limit` polls
// (each poll may itself suspend for a hardware-chosen interval).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) completing on `bar` with a transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ---- 5th-generation tensor cores (tcgen05) and tensor memory --------------
// Round to TF32 (10 explicit mantissa bits, nearest, ties away) as an FP32
// value with the low 13 bits clear, so that a kind::tf32 MMA reads exactly
// this value and x - tf32r(x) is the exact remainder.  The conversion leaves
// those 13 bits unspecified; they are cleared here.
__device__ __forceinline__ float tf32r(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r & 0xFFFFE000u);
}
// Tensor-memory allocation by one full warp: writes the base address
// (lane 0, first column) to *slot.  ncols: a power of two >= 32.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Make this thread's generic-proxy shared-memory writes visible to the
// async proxy (tcgen05.mma operand reads, bulk copies).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Shared-memory matrix descriptor, K-major without swizzle: the operand is
// made of core matrices of 8 rows x 16 bytes (128 contiguous bytes); lbo =
// byte distance between core matrices adjacent along K, sbo = between
// core matrices adjacent along M (or N).  Bits 46-47 hold the descriptor
// version (1); base offset, LBO mode and swizzle mode are 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of a dense kind::tf32 MMA: FP32 accumulator, TF32
// A and B, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t M, uint32_t N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
// D[tmem] (+)= A[smem] * B[smem]^T, one K = 8 step, issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive once on *bar when every tcgen05 operation this thread issued so far
// has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 32 consecutive 32-bit columns of the warp's 32 tensor-memory lanes (one
// lane per thread); complete after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32], int o) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr + (uint32_t)o));
}
// Wait for this thread's tensor-memory loads.  The loaded registers are
// read-write operands, so no use of them is scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                   "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]),
                   "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]),
                   "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :
                 : "memory");
}

// Programmatic dependent launch, first statement of a kernel launched with
// launch_pdl: wait until the previous grid in the stream has completed and
// its writes are visible.  The next grid's launch is triggered implicitly
// as this grid's CTAs exit, which still overlaps its launch with this
// grid's tail.  (Triggering at the start let the next grid's CTAs take up
// residence and wait beside long grids of small blocks, and slowed the LQR
// scans at T = 65536 from 528 to 793 us; the all-pairs kernels, which place
// their own trigger, were unaffected either way.)
__device__ __forceinline__ void pdl_prologue() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Split ticket of a CTA whose threads wrote partials before a CTA barrier:
// one thread's acquire-release atomic add at GPU scope publishes them
// (release, cumulative over the barrier) and, for the CTA that draws the
// last ticket, makes the other CTAs' partials visible to the reads that
// follow its next barrier (acquire) -- the ordering of a fence on each side
// of a relaxed atomic, in one operation.
__device__ __forceinline__ unsigned ticket_add(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Asynchronous global->shared copies (cp.async, 8 or 4 bytes): the next
// sub-block of per-step matrices of the Riccati kernels streams in while the
// current one is processed, and an input that only an epilogue reads is
// fetched at the start of a CTA without holding a register through its loop.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// Wait until at most G of this thread's committed groups are still in flight.
template <int G>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(G) : "memory");
}

// L2-coherent loads for data written by other CTAs of the same launch.
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }

__device__ __forceinline__ bool finitef(float x) { return fabsf(x) <= 3.402823466e38f; }

}  // namespace cov
