// lse_tc.cuh -- the fixed-offset Sinkhorn updates (M_GO) with the exponent
// matrix on the 5th-generation tensor cores.  Included by field.cu (it uses
// PairArgs, PairLaunch, the epilogue and the split merge defined there).
//
// For one CTA of 128 rows and a tile of kTcCols (256) columns the base-2 exponent,
// minus the row's fixed offset o_i (the previous log-sum-exp of the row),
//     w_ij - o_i = h_j + 2 xhat_i . yhat_j - o_i,
// is a rank-(d + 2) contraction.  It is computed exactly enough in FP32
// arithmetic by two kind::tf32 MMAs (M = 128, N = kTcCols, K = 8 each) from
// operands split into TF32 parts (v = v_hi + v_lo, and three parts for the
// large terms h_j and o_i, which makes them exact):
//   K slots 0-7  (coordinate record, constant over the iteration):
//     row    (X0h, X0h, X0l, X1h, X1h, X1l, X2h, X2h)     X = 2 xhat_i
//     column (C0h, C0l, C0h, C1h, C1l, C1h, C2h, C2l)     C = yhat_j
//   K slots 8-11 (h record, rewritten by every update's epilogue):
//     row    (1, 1, 1, X2l)
//     column (Hh, Hm, Hl, C2h)                           H = h_j
//   K slots 12-15 (constant ones on the column side):
//     row    (-Oh, -Om, -Ol, 0)                          O = o_i
//     column (1, 1, 1, 0)
// (unused coordinate slots are zero for d < 3).  Each product of two TF32
// values is exact; the dropped lo x lo products are below 2^-21 of the
// largest coordinate product.
//
// The accumulator (128 lanes x kTcCols FP32 columns) lands in tensor
// memory, double buffered.  Warp roles: the last warp allocates tensor
// memory, streams the column records through a shared-memory ring with the
// bulk-copy engine and issues the MMAs (one thread); the kTcSoftWarps reader
// warps take the accumulator with tcgen05.ld (warp w reads lanes
// 32 (w % 4) .. +31, i.e. rows, and columns 64 (w / 4) .. +63 of each tile)
// and fold 2^(w - o) into their row sums: one MUFU.EX2 and one add per pair,
// nothing else on the CUDA cores.
//
// Guards as in the CUDA-core M_GO kernel: a CTA whose partial exceeds 2^100
// (or is not finite) recomputes its columns with the running maximum on the
// CUDA cores; a row block whose merged sum is below 2^-60 is recomputed over
// all columns the same way.  Every wait is bounded (status bit kDevTimeout).
#pragma once

#include "tc_records.cuh"

namespace cov {

struct __align__(1024) TcSmem {
    float b0[kTcStages][kTcCols * kTcRecC];  // coordinate records of the tile's columns
    float bh[kTcStages][kTcCols * kTcRecH];  // h records
    float ones[kTcCols * kTcRecH];           // (1, 1, 1, 0): partner of the -o_i slots
    float a0[kTcRows * 8];                   // row slots 0-7
    float a1[kTcRows * 8];                   // row slots 8-15
    uint64_t full[kTcStages], empty[kTcStages], tfull[2], tempty[2], done;
    uint32_t tmem;
    int flag;
    int last;
    float red_m[2][kTcRows], red_s[kTcColGroups > 2 ? kTcColGroups : 2][kTcRows];
    float fin_m[kTcRows], fin_s[kTcRows];
};

// CUDA-core pass with the running maximum over the columns [cb, ce) for the
// CTA's 128 rows (two threads per row, one per half of the range), the same
// arithmetic as the CUDA-core kernel: w = h_j + sum_k X_k c_kj (FMA chain).
// Result (m, s) per row in S.fin_m / S.fin_s.  All threads call it.
template <int D>
__device__ void tc_cuda_core_pass(const PairArgs& a, TcSmem& S, int row0, int cb, int ce) {
    const int tid = threadIdx.x;
    if (tid < 2 * kTcRows) {
        const int r = tid & (kTcRows - 1), hf = tid / kTcRows;
        const int i = row0 + r;
        float X[D];
#pragma unroll
        for (int k = 0; k < D; ++k) X[k] = 2.0f * a.rows[(size_t)k * a.row_ld + i];
        const int mid = min(ce, cb + (((ce - cb) / 2 + 7) & ~7));
        const int jb = hf ? mid : cb, je = hf ? ce : mid;
        float m = kNegBig, s = 0.f;
        for (int j = jb; j < je; ++j) {
            float w = a.colh[j];
#pragma unroll
            for (int k = 0; k < D; ++k) w = fmaf(X[k], a.cols[(size_t)k * a.col_ld + j], w);
            if (w > m) {
                s = s * ex2(m - w) + 1.f;
                m = w;
            } else {
                s += ex2(w - m);
            }
        }
        S.red_m[hf][r] = m;
        S.red_s[hf][r] = s;
    }
    __syncthreads();
    if (tid < kTcRows) {
        float m = S.red_m[0][tid], s = S.red_s[0][tid];
        merge_into<D, M_G>(m, s, nullptr, S.red_m[1][tid], S.red_s[1][tid], nullptr);
        S.fin_m[tid] = m;
        S.fin_s[tid] = s;
    }
    __syncthreads();
}

template <int D>
__global__ void __launch_bounds__(kTcThreads, kTcMinBlocks) lse_tc_kernel(const __grid_constant__ PairLaunch L) {
    static_assert(D >= 1 && D <= 3, "tensor-core exponent layout covers d <= 3");
    __shared__ TcSmem S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int segi = ((int)blockIdx.x >= L.ctas0) ? 1 : 0;
    const PairArgs& a = segi ? L.seg[1] : L.seg[0];
    const int lb = (int)blockIdx.x - (segi ? L.ctas0 : 0);
    const int rb = lb / a.splits, sp = lb % a.splits;
    const int row0 = rb * kTcRows;
    // the column range is a whole number of tiles (planned in multiples of
    // kTcCols; records are padded with neutral columns)
    const int c0 = sp * a.cols_per_split;
    const int c1 = min(c0 + a.cols_per_split, a.n_cols8);
    const int nt = c1 > c0 ? (c1 - c0) / kTcCols : 0;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        mbar_init(&S.tfull[0], 1);
        mbar_init(&S.tfull[1], 1);
        mbar_init(&S.tempty[0], kTcSoftWarps);
        mbar_init(&S.tempty[1], kTcSoftWarps);
        mbar_init(&S.done, 1);
        S.flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kTcSoftWarps) tmem_alloc(&S.tmem, kTcTmemCols);
    for (int e = tid; e < kTcCols * kTcRecH; e += kTcThreads) S.ones[e] = (e & 3) < 3 ? 1.f : 0.f;
    if (!a.pre_ok) grid_dep_wait();
    // A operand: the rows' coordinates (constant) and fixed offsets (written
    // at least two launches back, so readable before the dependency wait)
    if (tid < kTcRows) {
        const int r = tid, i = row0 + r;
        float X[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < D; ++k) X[k] = 2.0f * a.rows[(size_t)k * a.row_ld + i];
        const float o = a.oca * a.oa[i] + (a.ob ? a.ocb * a.ob[i] : 0.f) + a.oc0;
        S.fin_m[r] = o;
        float s0[8], s1[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) s0[k] = s1[k] = 0.f;
#pragma unroll
        for (int k = 0; k < (D < 2 ? D : 2); ++k) {
            const float hi = tf32r(X[k]);
            s0[3 * k] = hi;
            s0[3 * k + 1] = hi;
            s0[3 * k + 2] = tf32r(X[k] - hi);
        }
        if constexpr (D == 3) {
            const float hi = tf32r(X[2]);
            s0[6] = hi;
            s0[7] = hi;
            s1[3] = tf32r(X[2] - hi);
        }
        s1[0] = s1[1] = s1[2] = 1.f;
        const float no = -o;
        s1[4] = tf32r(no);
        s1[5] = tf32r(no - s1[4]);
        s1[6] = tf32r(no - s1[4] - s1[5]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            S.a0[tc_rec_index(r, k)] = s0[k];
            S.a1[tc_rec_index(r, k)] = s1[k];
        }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const long long spin = a.spin_limit;

    if (warp == kTcSoftWarps) {
        // ---- copies and MMAs (one thread) ---------------------------------
        if (lane == 0) {
            auto issue = [&](int t) {
                const int s = t % kTcStages;
                const size_t col = (size_t)c0 + (size_t)t * kTcCols;
                mbar_arrive_expect_tx(&S.full[s], kTcTileBytes);
                bulk_g2s(S.b0[s], a.rec0 + col * kTcRecC, kTcCols * kTcRecC * 4, &S.full[s]);
                bulk_g2s(S.bh[s], a.rech + col * kTcRecH, kTcCols * kTcRecH * 4, &S.full[s]);
            };
            // the h records were written by the previous launch
            if (a.pre_ok) grid_dep_wait();
            grid_dep_launch();
            int issued = 0;
            for (; issued < min(nt, kTcStages); ++issued) issue(issued);
            constexpr uint32_t idesc = idesc_tf32(kTcRows, kTcCols);
            const uint64_t da0 = smem_desc(smem_u32(S.a0), 128, 256);
            const uint64_t da1 = smem_desc(smem_u32(S.a1), 128, 256);
            const uint32_t ones = smem_u32(S.ones);
            bool ok = true;
            int t = 0;
            for (; t < nt; ++t) {
                const int s = t % kTcStages, b = t & 1;
                ok = mbar_wait_bounded(&S.full[s], (unsigned)((t / kTcStages) & 1), spin);
                if (ok && t >= 2) ok = mbar_wait_bounded(&S.tempty[b], (unsigned)(((t - 2) >> 1) & 1), spin);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kTcCols);
                const uint32_t bh = smem_u32(S.bh[s]);
                mma_tf32(d, da0, smem_desc(smem_u32(S.b0[s]), 128, 256), idesc, 0u);
                mma_tf32(d, da1, smem_desc(bh, ones - bh, 128), idesc, 1u);
                tc_commit(&S.tfull[b]);
                tc_commit(&S.empty[s]);
                if (t >= 1 && issued < nt) {
                    // refill the stage of tile t-1 (its MMAs completed long ago)
                    ok = mbar_wait_bounded(&S.empty[(t - 1) % kTcStages], (unsigned)(((t - 1) / kTcStages) & 1), spin);
                    if (!ok) break;
                    issue(issued++);
                }
            }
            // nothing may still write tensor memory (or arrive on a barrier)
            // once the CTA frees it and exits: wait for the MMAs, and on the
            // error path for the copies issued but never waited for, with a
            // limit of at least 2^20 polls even when the tile waits have none
            const long long drain = spin > (1LL << 20) ? spin : (1LL << 20);
            tc_commit(&S.done);
            ok = mbar_wait_bounded(&S.done, 0u, drain) && ok;
            if (!ok) {
                raise_status(a.status, kDevTimeout);
                S.flag = 1;
                for (int u = t; u < issued; ++u)
                    mbar_wait_bounded(&S.full[u % kTcStages], (unsigned)((u / kTcStages) & 1), drain);
            }
        }
        __syncwarp();
    } else {
        // ---- accumulator readers ------------------------------------------
        const int q = warp & 3, hf = warp >> 2;  // lane quarter, column group
        // eight independent scalar sums: one MUFU.EX2 and one FADD per pair,
        // with no register packing between them
        float acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = 0.f;
        // The two 32-column halves of a reader's 64 columns are loaded one
        // step ahead, so that the tensor-memory load latency hides behind
        // MUFU work: half 1 of tile t while half 0 is summed, half 0 of tile
        // t + 1 (after its full barrier) while half 1 is summed.  pin() keeps
        // the sums between a load and its wait.
        auto pin = [&]() {
            asm volatile("" : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3]), "+f"(acc[4]), "+f"(acc[5]),
                         "+f"(acc[6]), "+f"(acc[7]));
        };
        // of the 64 values the last 2 kTcPolyPairs take 2^x on the FMA pipe
        // (exp2_fma2, two at a time), the rest MUFU.EX2
        auto sum32 = [&](const uint32_t (&v)[32], int base) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (base + j < 64 - 2 * kTcPolyPairs) acc[j & 7] += ex2(__uint_as_float(v[j]));
#pragma unroll
            for (int j = 0; j < 32; j += 2)
                if (base + j >= 64 - 2 * kTcPolyPairs) {
                    const float2 e = exp2_fma2(make_float2(__uint_as_float(v[j]), __uint_as_float(v[j + 1])));
                    acc[j & 7] += e.x;
                    acc[(j + 1) & 7] += e.y;
                }
        };
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hf * 64);
        uint32_t vA[32], vB[32];
        bool live = nt > 0;
        if (live) {
            const bool got = mbar_wait_bounded(&S.tfull[0], 0u, spin);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) {
                    raise_status(a.status, kDevTimeout);
                    S.flag = 1;
                }
                live = false;
            } else {
                tc_fence_after();
                tmem_ld32(tq, vA, 0);
                tmem_wait_ld(vA);
            }
        }
        for (int t = 0; live && t < nt; ++t) {
            const int b = t & 1;
            tmem_ld32(tq + (uint32_t)(b * kTcCols), vB, 32);
            pin();
            sum32(vA, 0);
            pin();
            tmem_wait_ld(vB);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.tempty[b]);
            const bool more = t + 1 < nt;
            if (more) {
                const bool got = mbar_wait_bounded(&S.tfull[b ^ 1], (unsigned)(((t + 1) >> 1) & 1), spin);
                if (!__all_sync(0xffffffffu, got)) {
                    if (lane == 0) {
                        raise_status(a.status, kDevTimeout);
                        S.flag = 1;
                    }
                    break;
                }
                tc_fence_after();
                tmem_ld32(tq + (uint32_t)((b ^ 1) * kTcCols), vA, 0);
            }
            pin();
            sum32(vB, 32);
            pin();
            if (more) tmem_wait_ld(vA);
        }
        S.red_s[hf][q * 32 + lane] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kTcSoftWarps) tmem_dealloc(tmem, kTcTmemCols);
    const bool timed_out = S.flag != 0;

    // ---- this CTA's partial (offset, sum) per row; overflow guard ---------
    bool over = false;
    if (tid < kTcRows) {
        float s = 0.f;
#pragma unroll
        for (int g = 0; g < kTcColGroups; ++g) s += S.red_s[g][tid];
        S.fin_s[tid] = s;
        over = row0 + tid < a.n_rows && !(s <= kOffsetHi);
    }
    if (__syncthreads_or(over) && !timed_out) tc_cuda_core_pass<D>(a, S, row0, c0, c1);

    if (a.splits > 1) {
        const size_t cs = (size_t)a.splits * a.part_ld;
        if (tid < kTcRows) {
            float* P = a.part + (size_t)sp * a.part_ld + row0 + tid;
            P[0] = S.fin_m[tid];
            P[cs] = S.fin_s[tid];
        }
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = ticket_add(&a.counters[rb], 1u);
            S.last = (prev == (unsigned)(a.splits - 1));
        }
        __syncthreads();
        if (!S.last) return;
        if (tid < kTcRows) {
            const int i = row0 + tid;
            float m = kNegBig, sv = 0.f;
            for (int p0 = 0; p0 < a.splits; p0 += 8) {
                float m2[8], s2[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const bool live = p0 + u < a.splits;
                    const float* P = a.part + (size_t)(live ? p0 + u : 0) * a.part_ld + i;
                    m2[u] = live ? ld_cg(P) : kNegBig;
                    s2[u] = live ? ld_cg(P + cs) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) merge_into<D, M_GO>(m, sv, nullptr, m2[u], s2[u], nullptr);
            }
            S.fin_m[tid] = m;
            S.fin_s[tid] = sv;
        }
        __syncthreads();
    }
    // a row whose sum is tiny may have lost terms to underflow
    bool tiny = false;
    if (tid < kTcRows) tiny = row0 + tid < a.n_rows && !(S.fin_s[tid] >= kOffsetLo);
    if (__syncthreads_or(tiny) && !timed_out) tc_cuda_core_pass<D>(a, S, row0, 0, a.n_cols8);
    if (tid < kTcRows) epilogue<D, M_GO>(a, row0 + tid, S.fin_m[tid], S.fin_s[tid], nullptr);
    if (a.splits > 1 && tid == 0) a.counters[rb] = 0u;  // ready for the next launch
}

// Coordinate and h records of the point sets (after the prep or a rescale):
// x -> c0x, hx -> hrx, hp and hp2 (both self-potential buffers) -> hrp and
// hrp2; y -> c0y, hy -> hry.  Padding points get zero coordinates and
// h = kPadH (their exponents vanish); the epilogues rewrite only the records
// of real points, so the padding of every record buffer is written here.
template <int D>
__global__ void tc_records_kernel(const float* __restrict__ xs, int Tp, const float* __restrict__ ys, int Mp,
                                  const float* __restrict__ hx, const float* __restrict__ hp,
                                  const float* __restrict__ hp2, const float* __restrict__ hy,
                                  float* __restrict__ c0x, float* __restrict__ c0y, float* __restrict__ hrx,
                                  float* __restrict__ hrp, float* __restrict__ hrp2, float* __restrict__ hry) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float c[3] = {0.f, 0.f, 0.f};
    float s[8];
    if (i < Tp) {
#pragma unroll
        for (int k = 0; k < D; ++k) c[k] = xs[(size_t)k * Tp + i];
        tc_crec<D>(c, s);
#pragma unroll
        for (int k = 0; k < 8; ++k) c0x[tc_rec_index(i, k)] = s[k];
        reinterpret_cast<float4*>(hrx)[i] = tc_hrec<D>(hx[i], c[2]);
        reinterpret_cast<float4*>(hrp)[i] = tc_hrec<D>(hp[i], c[2]);
        reinterpret_cast<float4*>(hrp2)[i] = tc_hrec<D>(hp2[i], c[2]);
    }
    if (i < Mp) {
#pragma unroll
        for (int k = 0; k < D; ++k) c[k] = ys[(size_t)k * Mp + i];
        tc_crec<D>(c, s);
#pragma unroll
        for (int k = 0; k < 8; ++k) c0y[tc_rec_index(i, k)] = s[k];
        reinterpret_cast<float4*>(hry)[i] = tc_hrec<D>(hy[i], c[2]);
    }
}

}  // namespace cov
