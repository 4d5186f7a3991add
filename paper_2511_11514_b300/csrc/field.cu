// field.cu -- the coverage flow fields of Sec. II-B on sm_103a:
//   * the Sinkhorn-divergence field (Eq. 5-7): log-domain Sinkhorn g-, f- and
//     debiasing p-updates and the barycentric gradient pass;
//   * the Stein variational field (Eq. 4) and the Gaussian-mixture score.
//
// All of them are one all-pairs kernel (`pairs_kernel`): a CTA holds 32*R
// rows in registers (R rows per lane, the same rows in each of its 4 warps),
// streams its slice of the column set through shared memory in tiles of 256
// columns with the bulk-copy engine (cp.async.bulk + mbarrier, double
// buffered), and each warp reduces a quarter of every tile.  Per pair the
// Sinkhorn modes evaluate, in base 2 with coordinates prescaled by
// 1/sqrt(eps ln 2),
//     w_ij = h_j + 2 xhat_i . yhat_j             (packed f32x2 FMA)
// and fold it into an online max-subtracted log-sum-exp (running maximum
// updated once per 8 columns with 3-input max instructions, the running sum
// rescaled by 2^(m_old - m_new) under a warp-uniform vote, 2^(w - m) on
// MUFU.EX2).
// The |xhat_i|^2 row term is constant along a row and is folded back into
// the potentials by the epilogue, so the Sinkhorn iteration runs entirely on
// the per-column terms h:
//     g-update (rows y, columns x):  hy_j = log2 b_j - LSE2_i(hx_i + 2 y.x)
//     f-update (rows x, columns y):  hx_i = log2 a   - LSE2_j(hy_j + 2 x.y)
//     p-update (rows x, columns x):  hp'_i = (log2 a + hp_i - LSE2_k(...))/2
// with hx = log2 a + f/(eps ln2) - |xhat|^2 etc.  Column splits of one row
// block are merged by the last CTA to finish (atomic ticket).
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "cov_device.cuh"
#include "cov_internal.h"
#include "tc_records.cuh"

namespace cov {

// M_GW: a log-sum-exp update (epilogue as M_G) that also writes the
// barycentric offset sum_j pi_ij (c_j - r_i) of its own softmax (the forward
// record the adjoint needs).
// M_GO: the same update as M_G with a FIXED per-row offset instead of a
// running maximum: the previous iteration's log-sum-exp of the row, o_i,
// which the new one differs from by little once the iteration has started,
//   LSE2_j(w_ij) = o_i + log2 sum_j 2^(w_ij - o_i)   (exact for any o_i).
// That drops the per-chunk maximum, compare and warp vote from the inner
// loop.  Guards: a CTA whose partial sum overflowed (> 2^100) redoes its
// columns with the running maximum; a row whose merged sum is tiny
// (< 2^-60, so terms may have flushed to zero) is recomputed over all
// columns with the running maximum by the merging CTA.
enum PairMode { M_G = 0, M_F = 1, M_P = 2, M_WY = 3, M_WX = 4, M_SVGD = 5, M_GW = 6, M_GO = 7, M_COUNT = 8 };

constexpr float kOffsetHi = 1.2676506e30f;   // 2^100
constexpr float kOffsetLo = 8.6736174e-19f;  // 2^-60

constexpr int kTile = 256;   // columns per staged tile
constexpr unsigned kRedoTicket = 1u << 16;  // split-ticket increment of a split that redid its columns
constexpr int kWarps = 4;    // warps per CTA, each takes a quarter of a tile
constexpr int kThreads = 32 * kWarps;
constexpr int kRowPad = 1024;  // point arrays are padded to this multiple
constexpr float kSvgdPad = 1.0e15f;  // SVGD padding coordinate (kernel -> 0)
// The one-launch Stein field for short trajectories (build flag
// -DCOV_SVGD_SMALL=0 takes the all-pairs kernel at every T).
#ifndef COV_SVGD_SMALL
#define COV_SVGD_SMALL 1
#endif

struct PairArgs {
    const float* rows;   // [D][row_ld]
    int row_ld;
    int n_rows;
    const float* cols;   // [D][col_ld]
    const float* colh;   // [col_ld] (Sinkhorn modes)
    const float* cols2;  // [D][col_ld] (SVGD: scaled score)
    int col_ld;
    int n_cols8;         // columns rounded up to 8 (padding holds neutral values)
    int cols_per_split;  // multiple of 8
    int splits;          // column splits of row blocks [0, n_hi); the others have splits - 1
    int n_hi;            // row blocks with `splits` splits (== n_rb: every row block)
    int cps_lo;          // columns per split of the row blocks with splits - 1
    float* part;         // [NACC][splits][part_ld]
    int part_ld;         // n_rb * rows per CTA
    unsigned* counters;  // [n_rb]
    int n_rb;            // row blocks of this segment
    int emode;           // log-sum-exp epilogue: M_G, M_F or M_P
    int pre_ok;          // rows and column coordinates were written before the previous launch
    float* out_h;
    const float* in_h;
    float log2a;
    // M_GO: row offset o_i = oca oa[i] + ocb ob[i] + oc0 (ob may be null);
    // fixed == 0 runs this segment with the running maximum instead
    const float* oa;
    const float* ob;
    float oca, ocb, oc0;
    int fixed;
    // tensor-core path (lse_tc.cuh): the columns' coordinate and h records;
    // out_rec (any log-sum-exp mode, may be null): the rows' h records,
    // rewritten with out_h for the next update that has these points as columns
    const float* rec0;
    const float* rech;
    float* out_rec;
    float* bary;         // [D][row_ld]
    float* a_out;        // [n_rows][D]
    float a_scale;
    unsigned* status;
    long long spin_limit;
};

template <int D, int MODE>
struct PairTraits {
    static constexpr bool kW = (MODE == M_WY || MODE == M_WX || MODE == M_GW);
    static constexpr bool kSV = (MODE == M_SVGD);
    static constexpr bool kO = (MODE == M_GO);
    static constexpr int NC = kSV ? 2 * D : D + 1;             // staged components per column
    static constexpr int NACC = kSV ? D : (kW ? 2 + D : 2);    // partial components per row
};

// Accumulator state of one row.
template <int D, bool kW, bool kSV>
struct RowAcc {
    float m;          // running max (Sinkhorn)
    float2 s;         // running sum (two packed halves)
    float2 acc[D];    // weighted sums (W and SVGD modes)
};

template <int D, int R, int MODE>
__device__ __forceinline__ void tile_compute(const float* __restrict__ st, int jb, int je,
                                             const float (&X)[R][D], const float (&Xr)[R][D],
                                             RowAcc<D, PairTraits<D, MODE>::kW, PairTraits<D, MODE>::kSV> (&ra)[R]) {
    using TR = PairTraits<D, MODE>;
#pragma unroll 1
    for (int j = jb; j < je; j += 8) {
        float c[TR::NC][8];
#pragma unroll
        for (int k = 0; k < TR::NC; ++k) {
            const float4 v0 = *reinterpret_cast<const float4*>(st + k * kTile + j);
            const float4 v1 = *reinterpret_cast<const float4*>(st + k * kTile + j + 4);
            c[k][0] = v0.x; c[k][1] = v0.y; c[k][2] = v0.z; c[k][3] = v0.w;
            c[k][4] = v1.x; c[k][5] = v1.y; c[k][6] = v1.z; c[k][7] = v1.w;
        }
#pragma unroll
        for (int r = 0; r < (TR::kSV ? R : 0); ++r) {
            if constexpr (TR::kSV) {
                // k_ij = 2^{-|xt_i - xt_j|^2};  acc += k (st_j - (xt_j - xt_i))
                float2 d2[4];
                float2 dx[D][4];
#pragma unroll
                for (int q = 0; q < 4; ++q) d2[q] = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const float2 xk = make_float2(X[r][k], X[r][k]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        dx[k][q] = sub2(make_float2(c[k][2 * q], c[k][2 * q + 1]), xk);
                        d2[q] = fma2(dx[k][q], dx[k][q], d2[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 e = make_float2(ex2(-d2[q].x), ex2(-d2[q].y));
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        ra[r].acc[k] = fma2(e, sub2(make_float2(c[D + k][2 * q], c[D + k][2 * q + 1]), dx[k][q]),
                                            ra[r].acc[k]);
                }
            }
        }
        if constexpr (TR::kO) {
            // fixed offset (held in m): 2^(w - o), no maximum
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) w[q] = make_float2(c[D][2 * q], c[D][2 * q + 1]);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const float2 xk = make_float2(X[r][k], X[r][k]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) w[q] = fma2(xk, make_float2(c[k][2 * q], c[k][2 * q + 1]), w[q]);
                }
                const float2 oo = make_float2(ra[r].m, ra[r].m);
                float2 e[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 dd = sub2(w[q], oo);
                    e[q] = make_float2(ex2(dd.x), ex2(dd.y));
                }
                ra[r].s = add2(ra[r].s, add2(add2(e[0], e[1]), add2(e[2], e[3])));
            }
        }
        if constexpr (!TR::kSV && !TR::kO) {
            // exponents of this chunk for all R rows, and each row's new running max
            float2 w[R][4];
            float mn[R];
            bool grew = false;
#pragma unroll
            for (int r = 0; r < R; ++r) {
#pragma unroll
                for (int q = 0; q < 4; ++q) w[r][q] = make_float2(c[D][2 * q], c[D][2 * q + 1]);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const float2 xk = make_float2(X[r][k], X[r][k]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) w[r][q] = fma2(xk, make_float2(c[k][2 * q], c[k][2 * q + 1]), w[r][q]);
                }
                mn[r] = max3f(max3f(ra[r].m, w[r][0].x, w[r][0].y), max3f(w[r][1].x, w[r][1].y, w[r][2].x),
                              max3f(w[r][2].y, w[r][3].x, w[r][3].y));
                grew |= mn[r] > ra[r].m;
            }
            // rescale what was accumulated by 2^(m_old - m_new) only when some
            // row of the warp raised its maximum (rare after the first tiles);
            // the vote keeps the branch uniform across the warp
            if (__any_sync(0xffffffffu, grew)) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float sc = ex2(ra[r].m - mn[r]);
                    const float2 sc2 = make_float2(sc, sc);
                    ra[r].s = mul2(ra[r].s, sc2);
                    if constexpr (TR::kW) {
#pragma unroll
                        for (int k = 0; k < D; ++k) ra[r].acc[k] = mul2(ra[r].acc[k], sc2);
                    }
                    ra[r].m = mn[r];
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 mm = make_float2(ra[r].m, ra[r].m);
                float2 e[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 dd = sub2(w[r][q], mm);
                    e[q] = make_float2(ex2(dd.x), ex2(dd.y));
                }
                ra[r].s = add2(ra[r].s, add2(add2(e[0], e[1]), add2(e[2], e[3])));
                if constexpr (TR::kW) {
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float2 xr = make_float2(Xr[r][k], Xr[r][k]);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            ra[r].acc[k] = fma2(e[q], sub2(make_float2(c[k][2 * q], c[k][2 * q + 1]), xr),
                                                ra[r].acc[k]);
                    }
                }
            }
        }
    }
}

// Merge partial (m2, s2, acc2) into (m, s, acc).
template <int D, int MODE>
__device__ __forceinline__ void merge_into(float& m, float& s, float* acc, float m2, float s2, const float* acc2) {
    using TR = PairTraits<D, MODE>;
    if constexpr (TR::kSV) {
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] += acc2[k];
    } else {
        const float M = fmaxf(m, m2);
        const float a1 = ex2(m - M), a2 = ex2(m2 - M);
        s = s * a1 + s2 * a2;
        if constexpr (TR::kW) {
#pragma unroll
            for (int k = 0; k < D; ++k) acc[k] = acc[k] * a1 + acc2[k] * a2;
        }
        m = M;
    }
}

// Sum of the partial sums of row i over all column splits when every split
// summed against the same fixed offset: the sums alone, CH loaded at once
// (one L2 round trip for up to CH splits), added in split order into four
// interleaved accumulators (deterministic).
template <int CH>
__device__ __forceinline__ float sum_lse_splits(const float* part, size_t part_ld, int splits, int ns, int i) {
    const float* S = part + (size_t)splits * part_ld + i;  // the sum component of the layout
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    for (int p0 = 0; p0 < ns; p0 += CH) {
        float s2[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) s2[u] = p0 + u < ns ? ld_cg(S + (size_t)(p0 + u) * part_ld) : 0.f;
#pragma unroll
        for (int u = 0; u < CH; ++u) t[u & 3] += s2[u];
    }
    return (t[0] + t[1]) + (t[2] + t[3]);
}

// Merge the (max, sum) partials of row i over all column splits into
// (m, s): CH partials are loaded at once (one L2 round trip per CH splits),
// then one maximum and a sum of independent rescaled terms -- no serial
// max/rescale chain through the partials.
template <int CH>
__device__ __forceinline__ void merge_lse_splits(const float* part, size_t part_ld, int splits, int ns, int i,
                                                 float& m, float& s) {
    const size_t cs = (size_t)splits * part_ld;  // component stride of the layout (the plan's largest count)
    m = kNegBig;
    s = 0.f;
    for (int p0 = 0; p0 < ns; p0 += CH) {
        float m2[CH], s2[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const bool live = p0 + u < ns;
            const float* P = part + (size_t)(live ? p0 + u : 0) * part_ld + i;
            m2[u] = live ? ld_cg(P) : kNegBig;
            s2[u] = live ? ld_cg(P + cs) : 0.f;
        }
        float M = m;
#pragma unroll
        for (int u = 0; u < CH; ++u) M = fmaxf(M, m2[u]);
        float t[4] = {s * ex2(m - M), 0.f, 0.f, 0.f};
#pragma unroll
        for (int u = 0; u < CH; ++u) t[u & 3] = fmaf(s2[u], ex2(m2[u] - M), t[u & 3]);
        s = (t[0] + t[1]) + (t[2] + t[3]);
        m = M;
    }
}

// `hin`, when given, holds a.in_h[i] (fetched early by the caller).
template <int D, int MODE>
__device__ __forceinline__ void epilogue(const PairArgs& a, int i, float m, float s, const float* acc,
                                         const float* hin = nullptr) {
    using TR = PairTraits<D, MODE>;
    if (i >= a.n_rows) return;
    bool ok = true;
    if constexpr (TR::kSV) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float v = a.a_out ? a.a_scale * acc[k] : 0.f;
            ok &= finitef(v);
            a.a_out[(size_t)i * D + k] = v;
        }
    } else if constexpr (MODE == M_WY) {
        const float inv = 1.0f / s;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float v = acc[k] * inv;
            ok &= finitef(v);
            a.bary[(size_t)k * a.row_ld + i] = v;
        }
    } else if constexpr (MODE == M_WX) {
        const float inv = 1.0f / s;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float v = a.a_scale * (a.bary[(size_t)k * a.row_ld + i] - acc[k] * inv);
            ok &= finitef(v);
            a.a_out[(size_t)i * D + k] = v;
        }
    } else {
        const float L = m + log2f(s);
        float v;
        if (a.emode == M_G) v = (hin ? *hin : a.in_h[i]) - L;
        else if (a.emode == M_F) v = a.log2a - L;
        else v = 0.5f * (a.log2a + (hin ? *hin : a.in_h[i]) - L);
        ok &= finitef(v);
        a.out_h[i] = v;
        if (a.out_rec)
            reinterpret_cast<float4*>(a.out_rec)[i] = tc_hrec<D>(v, D == 3 ? a.rows[(size_t)2 * a.row_ld + i] : 0.f);
        if constexpr (MODE == M_GW) {
            if (a.bary) {
                const float inv = 1.0f / s;
#pragma unroll
                for (int k = 0; k < D; ++k) a.bary[(size_t)k * a.row_ld + i] = acc[k] * inv;
            }
        }
    }
    if (!ok) raise_status(a.status, kDevNonfinite);
}

// One launch covers up to two independent passes ("segments", e.g. the
// g-update and the self p-update of the same Sinkhorn iteration): CTAs
// [0, ctas0) belong to seg[0], the rest to seg[1].
struct PairLaunch {
    PairArgs seg[2];
    int ctas0;
};

// Programmatic dependent launch: wait for the previous grid's results, and
// let the next grid start its prologue while this one runs.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Resident CTAs per SM the weighted (barycentre) modes are compiled for
// (build flag; 1 leaves the register count to the compiler).
#ifndef COV_BARY_MINB
#define COV_BARY_MINB 1
#endif
// Rows per thread of the weighted modes (build flag; 0: the context's setting).
#ifndef COV_BARY_R
#define COV_BARY_R 0
#endif
template <int MODE>
struct PairMinBlocks {
    static constexpr int value = (MODE == M_WY || MODE == M_WX || MODE == M_GW) ? COV_BARY_MINB : 1;
};

template <int D, int R, int MODE>
__global__ void __launch_bounds__(kThreads, PairMinBlocks<MODE>::value) pairs_kernel(const __grid_constant__ PairLaunch L) {
    using TR = PairTraits<D, MODE>;
    constexpr int NC = TR::NC;
    constexpr int NACC = TR::NACC;
    constexpr int RB = 32 * R;  // rows per CTA
    __shared__ __align__(128) float sm[2][NC * kTile];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red[kWarps][NACC][RB];
    __shared__ float epi_h[TR::kO ? RB : 1];  // the rows' in_h, for the epilogue
    __shared__ int s_last;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int segi = ((int)blockIdx.x >= L.ctas0) ? 1 : 0;
    const PairArgs a = segi ? L.seg[1] : L.seg[0];
    const int lb = (int)blockIdx.x - (segi ? L.ctas0 : 0);
    // this CTA's row block, split index, the row block's split count and
    // its columns (a plan may give some row blocks one split fewer)
    int rb, sp, ns, cps;
    if (lb < a.n_hi * a.splits) {
        rb = lb / a.splits;
        sp = lb % a.splits;
        ns = a.splits;
        cps = a.cols_per_split;
    } else {
        const int l2 = lb - a.n_hi * a.splits;
        ns = a.splits - 1;
        rb = a.n_hi + l2 / ns;
        sp = l2 % ns;
        cps = a.cps_lo;
    }
    const int row0 = rb * RB;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (!a.pre_ok) grid_dep_wait();

    float X[R][D], Xr[R][D];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float v = a.rows[(size_t)k * a.row_ld + row0 + r * 32 + lane];
            X[r][k] = TR::kSV ? v : 2.0f * v;
            Xr[r][k] = v;
        }
    RowAcc<D, TR::kW, TR::kSV> ra[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ra[r].m = kNegBig;
        ra[r].s = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < D; ++k) ra[r].acc[k] = make_float2(0.f, 0.f);
    }

    const bool fixed = TR::kO && a.fixed;
    if (fixed) {
        // the fixed offsets: the previous iteration's log-sum-exp of each row
        // (written two launches ago, so readable before the dependency wait)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = row0 + r * 32 + lane;
            ra[r].m = a.oca * a.oa[i] + (a.ob ? a.ocb * a.ob[i] : 0.f) + a.oc0;
        }
    }

    const int c0 = sp * cps;
    const int c1 = min(c0 + cps, a.n_cols8);
    __syncthreads();

    // A tile is the column coordinates (constant over the Sinkhorn loop) and
    // the per-column term h (written by the previous launch).
    auto issue_coords = [&](int cb, int ce, int t, int stg) {
        const int tc = cb + t * kTile;
        const int nc = min(kTile, ce - tc);
        const unsigned bytes = (unsigned)nc * 4u;
        mbar_arrive_expect_tx(&bar[stg], bytes * NC);
#pragma unroll
        for (int k = 0; k < D; ++k) bulk_g2s(&sm[stg][k * kTile], a.cols + (size_t)k * a.col_ld + tc, bytes, &bar[stg]);
    };
    auto issue_h = [&](int cb, int ce, int t, int stg) {
        const int tc = cb + t * kTile;
        const int nc = min(kTile, ce - tc);
        const unsigned bytes = (unsigned)nc * 4u;
        if constexpr (TR::kSV) {
#pragma unroll
            for (int k = 0; k < D; ++k)
                bulk_g2s(&sm[stg][(D + k) * kTile], a.cols2 + (size_t)k * a.col_ld + tc, bytes, &bar[stg]);
        } else {
            bulk_g2s(&sm[stg][D * kTile], a.colh + tc, bytes, &bar[stg]);
        }
    };

    // The epilogue's per-row input (log2 b of a g-update, the previous
    // potential of a p-update) is copied to shared memory once the
    // dependency wait has passed, so that the merging CTA does not start an
    // L2 round trip of its own after the merge; each thread later reads the
    // rows it copied itself.
    const bool epi_pre = TR::kO && a.in_h && a.emode != M_F;
    auto prefetch_epi = [&]() {
        if constexpr (TR::kO) {
            if (epi_pre) {
                for (int q = threadIdx.x; q < RB; q += kThreads)
                    if (row0 + q < a.n_rows) cp_async4(&epi_h[q], a.in_h + row0 + q);
                cp_async_commit();
            }
        }
    };

    // One pass over the columns [cb, ce).  Tiles alternate between the two
    // stages by a running count over all passes (which also gives each
    // mbarrier's phase parity).  The first pass overlaps its first column
    // copies with the previous launch (programmatic dependent launch).
    int gtile = 0;
    bool timed_out = false;
    auto run_pass = [&](int cb, int ce, bool first, bool fixed) {
        const int nt = ce > cb ? (ce - cb + kTile - 1) / kTile : 0;
        if (first) {
            if (threadIdx.x == 0 && nt > 0) issue_coords(cb, ce, 0, gtile & 1);
            if (a.pre_ok) grid_dep_wait();
            grid_dep_launch();
            if (threadIdx.x == 0 && nt > 0) issue_h(cb, ce, 0, gtile & 1);
            prefetch_epi();
        } else if (threadIdx.x == 0 && nt > 0) {
            issue_coords(cb, ce, 0, gtile & 1);
            issue_h(cb, ce, 0, gtile & 1);
        }
        int bad_tile = -1;
        for (int t = 0; t < nt; ++t) {
            const int g = gtile + t, stg = g & 1;
            if (threadIdx.x == 0 && t + 1 < nt) {
                issue_coords(cb, ce, t + 1, stg ^ 1);
                issue_h(cb, ce, t + 1, stg ^ 1);
            }
            const bool ok = mbar_wait_bounded(&bar[stg], (unsigned)((g >> 1) & 1), a.spin_limit);
            if (__syncthreads_or(!ok)) {
                bad_tile = t;
                break;
            }
            const int nc = min(kTile, ce - (cb + t * kTile));
            const int per = ((nc / 8 + kWarps - 1) / kWarps) * 8;
            const int jb = min(nc, warp * per), je = min(nc, jb + per);
            if constexpr (TR::kO) {
                if (fixed)
                    tile_compute<D, R, M_GO>(sm[stg], jb, je, X, Xr, ra);
                else
                    tile_compute<D, R, M_G>(sm[stg], jb, je, X, Xr, ra);
            } else {
                tile_compute<D, R, MODE>(sm[stg], jb, je, X, Xr, ra);
            }
            __syncthreads();
        }
        if (bad_tile >= 0) {
            // A tile never arrived: record it, drain the copies still in
            // flight (bounded) so no bulk copy lands after the CTA exits, and
            // fall through with whatever was accumulated (the status marks it
            // invalid); no further pass runs.
            if (threadIdx.x == 0) {
                raise_status(a.status, kDevTimeout);
                const long long drain = a.spin_limit > (1LL << 20) ? a.spin_limit : (1LL << 20);
                const int g = gtile + bad_tile;
                mbar_wait_bounded(&bar[g & 1], (unsigned)((g >> 1) & 1), drain);
                if (bad_tile + 1 < nt) mbar_wait_bounded(&bar[(g + 1) & 1], (unsigned)(((g + 1) >> 1) & 1), drain);
            }
            timed_out = true;
            __syncthreads();
        }
        gtile += nt;
    };
    run_pass(c0, c1, true, fixed);

    if constexpr (TR::kO) {
        __shared__ float fin_m[RB], fin_s[RB];
        auto reset_rows = [&]() {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ra[r].m = kNegBig;
                ra[r].s = make_float2(0.f, 0.f);
            }
        };
        // a partial that overflowed: redo this CTA's columns with the running maximum
        bool over = false;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (fixed && row0 + r * 32 + lane < a.n_rows) over |= !(ra[r].s.x + ra[r].s.y <= kOffsetHi);
        const bool redid = __syncthreads_or(over) && !timed_out;
        if (redid) {
            reset_rows();
            run_pass(c0, c1, false, false);
        }
        // the 4 warps' (m, s) of each row -> fin
        auto reduce_warps = [&]() {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                red[warp][0][r * 32 + lane] = ra[r].m;
                red[warp][1][r * 32 + lane] = ra[r].s.x + ra[r].s.y;
            }
            __syncthreads();
            for (int q = threadIdx.x; q < RB; q += kThreads) {
                float m = red[0][0][q], sv = red[0][1][q];
#pragma unroll
                for (int w = 1; w < kWarps; ++w) merge_into<D, MODE>(m, sv, nullptr, red[w][0][q], red[w][1][q], nullptr);
                fin_m[q] = m;
                fin_s[q] = sv;
            }
            __syncthreads();
        };
        reduce_warps();
        if (ns > 1) {
            const size_t cs = (size_t)a.splits * a.part_ld;
            for (int q = threadIdx.x; q < RB; q += kThreads) {
                float* P = a.part + (size_t)sp * a.part_ld + row0 + q;
                P[0] = fin_m[q];
                P[cs] = fin_s[q];
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                // the ticket also counts, above bit 16, the splits that redid
                // their columns with the running maximum
                const unsigned add = 1u + (redid ? kRedoTicket : 0u);
                const unsigned prev = ticket_add(&a.counters[rb], add);
                s_last = (prev & (kRedoTicket - 1u)) != (unsigned)(ns - 1) ? 0 : (prev + add >= kRedoTicket ? 2 : 1);
            }
            __syncthreads();
            if (!s_last) {
                if (epi_pre) cp_async_wait_all();  // no copy lands after the CTA exits
                return;
            }
            // every split against the same fixed offset (this CTA's fin_m):
            // a plain sum; otherwise the general merge
            const bool plain = fixed && s_last == 1;
            for (int q = threadIdx.x; q < RB; q += kThreads) {
                if (plain) {
                    fin_s[q] = sum_lse_splits<32>(a.part, (size_t)a.part_ld, a.splits, ns, row0 + q);
                } else {
                    float m, sv;
                    merge_lse_splits<16>(a.part, (size_t)a.part_ld, a.splits, ns, row0 + q, m, sv);
                    fin_m[q] = m;
                    fin_s[q] = sv;
                }
            }
            __syncthreads();
        }
        // a row whose sum is tiny may have lost terms to underflow: recompute
        // the whole row block over all columns with the running maximum
        bool tiny = false;
        for (int q = threadIdx.x; q < RB; q += kThreads)
            if (fixed && row0 + q < a.n_rows) tiny |= !(fin_s[q] >= kOffsetLo);
        if (__syncthreads_or(tiny) && !timed_out) {
            reset_rows();
            run_pass(0, a.n_cols8, false, false);
            reduce_warps();
        }
        if (epi_pre) cp_async_wait_all();
        for (int q = threadIdx.x; q < RB; q += kThreads)
            epilogue<D, MODE>(a, row0 + q, fin_m[q], fin_s[q], nullptr, epi_pre ? &epi_h[q] : nullptr);
        if (ns > 1 && threadIdx.x == 0) a.counters[rb] = 0u;  // ready for the next launch
        return;
    }

    // ---- reduce the 4 warps' partials of each row in shared memory ----------
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int q = r * 32 + lane;
        if constexpr (TR::kSV) {
#pragma unroll
            for (int k = 0; k < D; ++k) red[warp][k][q] = ra[r].acc[k].x + ra[r].acc[k].y;
        } else {
            red[warp][0][q] = ra[r].m;
            red[warp][1][q] = ra[r].s.x + ra[r].s.y;
            if constexpr (TR::kW) {
#pragma unroll
                for (int k = 0; k < D; ++k) red[warp][2 + k][q] = ra[r].acc[k].x + ra[r].acc[k].y;
            }
        }
    }
    __syncthreads();
    constexpr int KA = TR::kSV ? D : (TR::kW ? D : 1);
    for (int q = threadIdx.x; q < RB; q += kThreads) {
        float m, s, acc[KA];
        if constexpr (TR::kSV) {
            m = 0.f;
            s = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) acc[k] = red[0][k][q];
        } else {
            m = red[0][0][q];
            s = red[0][1][q];
            if constexpr (TR::kW) {
#pragma unroll
                for (int k = 0; k < D; ++k) acc[k] = red[0][2 + k][q];
            }
        }
#pragma unroll
        for (int w = 1; w < kWarps; ++w) {
            float a2[KA];
            float m2 = 0.f, s2 = 0.f;
            if constexpr (TR::kSV) {
#pragma unroll
                for (int k = 0; k < D; ++k) a2[k] = red[w][k][q];
            } else {
                m2 = red[w][0][q];
                s2 = red[w][1][q];
                if constexpr (TR::kW) {
#pragma unroll
                    for (int k = 0; k < D; ++k) a2[k] = red[w][2 + k][q];
                }
            }
            merge_into<D, MODE>(m, s, acc, m2, s2, a2);
        }
        const int i = row0 + q;
        if (ns == 1) {
            epilogue<D, MODE>(a, i, m, s, acc);
        } else {
            float* P = a.part + (size_t)sp * a.part_ld + i;
            const size_t cs = (size_t)a.splits * a.part_ld;  // component stride
            if constexpr (TR::kSV) {
#pragma unroll
                for (int k = 0; k < D; ++k) P[k * cs] = acc[k];
            } else {
                P[0] = m;
                P[cs] = s;
                if constexpr (TR::kW) {
#pragma unroll
                    for (int k = 0; k < D; ++k) P[(2 + k) * cs] = acc[k];
                }
            }
        }
    }
    if (ns == 1) return;

    // ---- last CTA of this row block merges the splits ------------------------
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = ticket_add(&a.counters[rb], 1u);
        s_last = (prev == (unsigned)(ns - 1));
    }
    __syncthreads();
    if (!s_last) return;
    const size_t cs = (size_t)a.splits * a.part_ld;
    for (int q = threadIdx.x; q < RB; q += kThreads) {
        const int i = row0 + q;
        if constexpr (!TR::kW && !TR::kSV) {
            float m, s;
            merge_lse_splits<16>(a.part, (size_t)a.part_ld, a.splits, ns, i, m, s);
            epilogue<D, MODE>(a, i, m, s, nullptr);
            continue;
        }
        float m = kNegBig, s = 0.f, acc[KA];
#pragma unroll
        for (int k = 0; k < KA; ++k) acc[k] = 0.f;
        // splits in groups of 8: all loads of a group are issued before the
        // first merge, so the L2 round trips overlap instead of serialising
        for (int p0 = 0; p0 < ns; p0 += 8) {
            float m2[8], s2[8], a2[8][KA];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool live = p0 + u < ns;
                const float* P = a.part + (size_t)(live ? p0 + u : 0) * a.part_ld + i;
                m2[u] = kNegBig;
                s2[u] = 0.f;
#pragma unroll
                for (int k = 0; k < KA; ++k) a2[u][k] = 0.f;
                if (live) {
                    if constexpr (TR::kSV) {
#pragma unroll
                        for (int k = 0; k < D; ++k) a2[u][k] = ld_cg(P + k * cs);
                    } else {
                        m2[u] = ld_cg(P);
                        s2[u] = ld_cg(P + cs);
                        if constexpr (TR::kW) {
#pragma unroll
                            for (int k = 0; k < D; ++k) a2[u][k] = ld_cg(P + (2 + k) * cs);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) merge_into<D, MODE>(m, s, acc, m2[u], s2[u], a2[u]);
        }
        epilogue<D, MODE>(a, i, m, s, acc);
    }
    if (threadIdx.x == 0) a.counters[rb] = 0u;  // ready for the next launch
}

}  // namespace cov

#include "lse_tc.cuh"

// ---------------------------------------------------------------------------
// Split planning: pick the number of column splits per row block that
// minimises (waves of CTAs) x (columns per CTA + fixed cost) + merge cost.
// Splits are whole multiples of `unit` columns.
// ---------------------------------------------------------------------------
cov::SplitPlan cov::plan_splits(int n_rows, int n_cols, int rows_per_cta, int slots, int unit, int fixed,
                                int max_waves) {
    SplitPlan best{};
    const int n_rb = (n_rows + rows_per_cta - 1) / rows_per_cta;
    const int units = (n_cols + unit - 1) / unit;
    const int smax = std::max(1, std::min(units, (max_waves * slots + n_rb - 1) / n_rb));
    double best_cost = 1e300;
    for (int s = 1; s <= smax; ++s) {
        const int cpu = (units + s - 1) / s;
        const int s_eff = (units + cpu - 1) / cpu;
        const long long ctas = (long long)n_rb * s_eff;
        const long long waves = (ctas + slots - 1) / slots;
        const double cost = (double)waves * ((double)cpu * unit + fixed) + (s_eff > 1 ? 4.0 * s_eff : 0.0);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = SplitPlan{n_rb, s_eff, cpu * unit};
        }
    }
    return best;
}

namespace cov {

// ---------------------------------------------------------------------------
// Prep kernels
// ---------------------------------------------------------------------------
// scal layout: [0..5] centre, [8] 1/sum(b) (or 0 when b == NULL)
//
// One CTA.  The points are read as float4 runs of the flat [M][d] array:
// with 960 threads a thread's run advances by 3840 floats, a multiple of
// every d <= 6, so lane e of each of its float4 loads holds component
// (4 tid + e) mod d and four running sums suffice; eight loads per thread
// are in flight at a time.  A pointer that is not 16-byte aligned, and the
// last few floats, take scalar loads.  Warp totals are added in warp order.
constexpr int kCentreThreads = 960;
constexpr int kCentreUnroll = 8;

__device__ __forceinline__ void add_component(float (&acc)[COV_MAX_D + 1], int c, float v) {
#pragma unroll
    for (int k = 0; k <= COV_MAX_D; ++k)
        if (k == c) acc[k] += v;
}

// Sum of n floats of p from flat index 0 as float4 runs (when aligned): the
// four lane sums of this thread, and the scalar tail added to acc[c(f)].
__device__ __forceinline__ size_t sum_runs(const float* __restrict__ p, size_t n, float (&ls)[4]) {
    const size_t nvec = (reinterpret_cast<uintptr_t>(p) & 15u) == 0 ? n / 4 : 0;
    const float4* p4 = reinterpret_cast<const float4*>(p);
    for (size_t q0 = threadIdx.x; q0 < nvec; q0 += (size_t)kCentreThreads * kCentreUnroll) {
        float4 v[kCentreUnroll];
#pragma unroll
        for (int u = 0; u < kCentreUnroll; ++u) {
            const size_t q = q0 + (size_t)u * kCentreThreads;
            v[u] = q < nvec ? p4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kCentreUnroll; ++u) {
            ls[0] += v[u].x;
            ls[1] += v[u].y;
            ls[2] += v[u].z;
            ls[3] += v[u].w;
        }
    }
    return 4 * nvec;  // first flat index left to the scalar tail
}

__global__ void __launch_bounds__(kCentreThreads) sk_centre_kernel(const float* __restrict__ y, int M, int d,
                                                                   const float* __restrict__ b,
                                                                   float* __restrict__ scal) {
    pdl_prologue();
    __shared__ float sh[kCentreThreads / 32][COV_MAX_D + 1];
    const int tid = threadIdx.x;
    float acc[COV_MAX_D + 1];
#pragma unroll
    for (int k = 0; k <= COV_MAX_D; ++k) acc[k] = 0.f;
    const size_t ny = (size_t)M * d;
    float ls[4] = {0.f, 0.f, 0.f, 0.f};
    const size_t ty = sum_runs(y, ny, ls);
#pragma unroll
    for (int e = 0; e < 4; ++e) add_component(acc, (4 * tid + e) % d, ls[e]);
    for (size_t f = ty + tid; f < ny; f += kCentreThreads) add_component(acc, (int)(f % (size_t)d), y[f]);
    if (b) {
        float lb[4] = {0.f, 0.f, 0.f, 0.f};
        const size_t tb = sum_runs(b, (size_t)M, lb);
        acc[COV_MAX_D] += (lb[0] + lb[1]) + (lb[2] + lb[3]);
        for (size_t f = tb + tid; f < (size_t)M; f += kCentreThreads) acc[COV_MAX_D] += b[f];
    }
#pragma unroll
    for (int k = 0; k <= COV_MAX_D; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    const int w = tid >> 5, l = tid & 31;
    if (l == 0)
#pragma unroll
        for (int k = 0; k <= COV_MAX_D; ++k) sh[w][k] = acc[k];
    __syncthreads();
    if (tid <= COV_MAX_D) {
        float t = 0.f;
        for (int i = 0; i < kCentreThreads / 32; ++i) t += sh[i][tid];
        if (tid < COV_MAX_D) scal[tid] = tid < d ? t / (float)M : 0.f;
        else scal[8] = b ? 1.0f / t : 0.f;
    }
}

struct SkBufs {
    float *xs, *ys, *hx, *hy, *hp0, *hp1, *lb, *nx, *ny, *bary, *scal, *part;
    // tensor-core records (tc_records.cuh; null when not carved): coordinate
    // records of x and y, h records of hx, hp (two buffers) and hy
    float *c0x, *c0y, *hrx, *hrp0, *hrp1, *hry;
    unsigned* counters;  // [M_COUNT][cnt_ld]
    int Tp, Mp, cnt_ld;
    size_t part_floats;
};

__global__ void sk_prep_kernel(const float* __restrict__ x, int x_ld, int T, const float* __restrict__ y, int M,
                               const float* __restrict__ b, int d, float inv_sigma, float inv_epsln2,
                               float log2a, int warm, const float* __restrict__ f, const float* __restrict__ g,
                               const float* __restrict__ p, SkBufs B, unsigned* status) {
    pdl_prologue();
    const float* c = B.scal;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B.Tp) {
        float n2 = 0.f;
        for (int k = 0; k < d; ++k) {
            const float v = i < T ? (x[(size_t)i * x_ld + k] - c[k]) * inv_sigma : 0.f;
            B.xs[(size_t)k * B.Tp + i] = v;
            n2 = fmaf(v, v, n2);
        }
        B.nx[i] = n2;
        if (i < T) {
            const float fh = warm ? f[i] * inv_epsln2 : 0.f;
            const float ph = warm ? p[i] * inv_epsln2 : 0.f;
            B.hx[i] = log2a + fh - n2;
            B.hp0[i] = log2a + ph - n2;
            if (!finitef(B.hx[i]) || !finitef(B.hp0[i])) raise_status(status, kDevNonfinite);
        } else {
            B.hx[i] = kPadH;
            B.hp0[i] = kPadH;
            B.hp1[i] = kPadH;
        }
    }
    if (i < B.Mp) {
        float n2 = 0.f;
        for (int k = 0; k < d; ++k) {
            const float v = i < M ? (y[(size_t)i * d + k] - c[k]) * inv_sigma : 0.f;
            B.ys[(size_t)k * B.Mp + i] = v;
            n2 = fmaf(v, v, n2);
        }
        B.ny[i] = n2;
        if (i < M) {
            const float lbj = b ? log2f(b[i] * c[8]) : -log2f((float)M);
            B.lb[i] = lbj;
            const float gh = warm ? g[i] * inv_epsln2 : 0.f;
            B.hy[i] = lbj + gh - n2;
            if (!finitef(B.hy[i])) raise_status(status, kDevNonfinite);
        } else {
            B.lb[i] = 0.f;
            B.hy[i] = kPadH;
        }
    }
}

__global__ void sk_finish_kernel(int T, int M, float epsln2, float log2a, SkBufs B, const float* __restrict__ hp,
                                 float* __restrict__ f, float* __restrict__ g, float* __restrict__ p,
                                 unsigned* status) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = true;
    if (i < T) {
        if (f) {
            const float v = (B.hx[i] - log2a + B.nx[i]) * epsln2;
            f[i] = v;
            ok &= finitef(v);
        }
        if (p) {
            const float v = (hp[i] - log2a + B.nx[i]) * epsln2;
            p[i] = v;
            ok &= finitef(v);
        }
    }
    if (i < M && g) {
        const float v = (B.hy[i] - B.lb[i] + B.ny[i]) * epsln2;
        g[i] = v;
        ok &= finitef(v);
    }
    if (!ok) raise_status(status, kDevNonfinite);
}

// eps-scaling stage change: every base-2 quantity depends on eps through the
// prescale xhat = (x - c)/sqrt(eps ln 2) and the potential units eps ln 2.
// Moving from eps_old to eps_new multiplies the coordinates by
// ratio = sqrt(eps_old/eps_new) and converts each potential term, e.g.
//   f/(eps_new ln2) = (hx - log2 a + |xhat_old|^2) eps_old/eps_new,
//   hx_new = log2 a + f/(eps_new ln2) - |xhat_new|^2  (likewise hy with log2 b, hp).
__global__ void sk_rescale_kernel(SkBufs B, int T, int M, int d, float ratio, float erat, float log2a,
                                  float* __restrict__ hp, unsigned* status) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = true;
    if (i < B.Tp) {
        float n2 = 0.f;
        for (int k = 0; k < d; ++k) {
            const float v = B.xs[(size_t)k * B.Tp + i] * ratio;
            B.xs[(size_t)k * B.Tp + i] = v;
            n2 = fmaf(v, v, n2);
        }
        const float n_old = B.nx[i];
        B.nx[i] = n2;
        if (i < T) {
            B.hx[i] = log2a + (B.hx[i] - log2a + n_old) * erat - n2;
            hp[i] = log2a + (hp[i] - log2a + n_old) * erat - n2;
            ok &= finitef(B.hx[i]) && finitef(hp[i]);
        }
    }
    if (i < B.Mp) {
        float n2 = 0.f;
        for (int k = 0; k < d; ++k) {
            const float v = B.ys[(size_t)k * B.Mp + i] * ratio;
            B.ys[(size_t)k * B.Mp + i] = v;
            n2 = fmaf(v, v, n2);
        }
        const float n_old = B.ny[i];
        B.ny[i] = n2;
        if (i < M) {
            B.hy[i] = B.lb[i] + (B.hy[i] - B.lb[i] + n_old) * erat - n2;
            ok &= finitef(B.hy[i]);
        }
    }
    if (!ok) raise_status(status, kDevNonfinite);
}

// eps of iteration t under the scaling schedule (the same product as the
// oracle's): max(eps, eps_start eps_decay^t); eps_start <= eps: no scaling.
static double anneal_eps(double eps, double eps_start, double eps_decay, int t) {
    double e = eps_start;
    for (int k = 0; k < t; ++k) e *= eps_decay;
    return e > eps ? e : eps;
}

// ---------------------------------------------------------------------------
// Launch dispatch.  Kernel families: M_G (log-sum-exp updates; the epilogue
// g/f/p is chosen per segment at run time), M_WY, M_WX, M_SVGD.  Launches use
// programmatic stream serialisation (PDL), so a launch's prologue overlaps
// the tail of the previous one; every kernel waits (griddepcontrol.wait)
// before it reads the previous launch's results or writes scratch.
// ---------------------------------------------------------------------------
// Resident CTAs per SM of one kernel instantiation (queried once).
template <int D, int R, int MODE>
static int occupancy_t() {
    static int occ = 0;
    if (occ == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, pairs_kernel<D, R, MODE>, kThreads, 0) != cudaSuccess ||
            v < 1) {
            cudaGetLastError();
            v = 1;
        }
        occ = v;
    }
    return occ;
}

// n_ctas > 0: launch; n_ctas == 0: return the resident CTAs per SM in *occ.
template <int D, int R, int MODE>
static cudaError_t launch_pairs_t(const PairLaunch& L, int n_ctas, cudaStream_t st, int* occ = nullptr) {
    if (occ) {
        *occ = occupancy_t<D, R, MODE>();
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)n_ctas);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pairs_kernel<D, R, MODE>, L);
}

template <int D, int R>
static cudaError_t launch_pairs_mode(int family, const PairLaunch& L, int n, cudaStream_t st, int* occ) {
    switch (family) {
        case M_G: return launch_pairs_t<D, R, M_G>(L, n, st, occ);
        case M_WY: return launch_pairs_t<D, R, M_WY>(L, n, st, occ);
        case M_WX: return launch_pairs_t<D, R, M_WX>(L, n, st, occ);
        case M_SVGD: return launch_pairs_t<D, R, M_SVGD>(L, n, st, occ);
        case M_GW: return launch_pairs_t<D, R, M_GW>(L, n, st, occ);
        case M_GO: return launch_pairs_t<D, R, M_GO>(L, n, st, occ);
    }
    return cudaErrorInvalidValue;
}

template <int D>
static cudaError_t launch_pairs_r(int R, int family, const PairLaunch& L, int n, cudaStream_t st, int* occ) {
    if constexpr (D == 2) {
        if (R == 2) return launch_pairs_mode<D, 2>(family, L, n, st, occ);
        if (R == 8) return launch_pairs_mode<D, 8>(family, L, n, st, occ);
    }
    return launch_pairs_mode<D, 4>(family, L, n, st, occ);
}

static cudaError_t launch_pairs_d(int d, int R, int family, const PairLaunch& L, int n, cudaStream_t st, int* occ) {
    switch (d) {
        case 1: return launch_pairs_r<1>(R, family, L, n, st, occ);
        case 2: return launch_pairs_r<2>(R, family, L, n, st, occ);
        case 3: return launch_pairs_r<3>(R, family, L, n, st, occ);
        case 4: return launch_pairs_r<4>(R, family, L, n, st, occ);
        case 5: return launch_pairs_r<5>(R, family, L, n, st, occ);
        case 6: return launch_pairs_r<6>(R, family, L, n, st, occ);
    }
    return cudaErrorInvalidValue;
}

template <int D>
static cudaError_t launch_tc_t(const PairLaunch& L, int n_ctas, cudaStream_t st, int* occ) {
    if (occ) {
        static int cached = 0;
        if (cached == 0) {
            // resident CTAs per SM from the kernel's own resources: registers
            // (allocated per warp in units of 256), static shared memory (plus
            // 1 KB the system reserves per CTA; largest carveout requested)
            // and tensor memory (512 columns per SM)
            cudaFuncSetAttribute(lse_tc_kernel<D>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
            cudaFuncAttributes fa{};
            int v = 1;
            if (cudaFuncGetAttributes(&fa, lse_tc_kernel<D>) == cudaSuccess && fa.numRegs > 0) {
                const int warps = kTcThreads / 32;
                const int regs_cta = warps * (((fa.numRegs * 32) + 255) / 256 * 256);
                const int by_regs = 65536 / regs_cta;
                const int by_smem = (228 * 1024) / ((int)fa.sharedSizeBytes + 1024);
                v = std::max(1, std::min(by_regs, by_smem));
            } else {
                cudaGetLastError();
            }
            cached = std::min(v, kTcMinBlocks);
        }
        *occ = cached;
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)n_ctas);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, lse_tc_kernel<D>, L);
}

static cudaError_t launch_tc_d(int d, const PairLaunch& L, int n, cudaStream_t st, int* occ) {
    switch (d) {
        case 1: return launch_tc_t<1>(L, n, st, occ);
        case 2: return launch_tc_t<2>(L, n, st, occ);
        case 3: return launch_tc_t<3>(L, n, st, occ);
    }
    return cudaErrorInvalidValue;
}

static int effective_R(int d, int R) { return (d == 2 && (R == 2 || R == 8)) ? R : 4; }

constexpr int kMaxSlots = 1536;           // CTA slots assumed by the workspace bound
constexpr size_t kPartRows = (size_t)2 * kMaxSlots * 256 + 256;

static int cnt_ld_for(int Tp, int Mp) { return std::max(Tp, Mp) / 64 + 1; }

static void plan_segment(PairArgs& a, int n_cols, int RB, int slots, unsigned* counters, int unit = 8,
                         int fixed = 64, int max_waves = 2) {
    const SplitPlan pl = plan_splits(a.n_rows, n_cols, RB, slots, unit, fixed, max_waves);
    a.n_cols8 = (int)round_up((size_t)n_cols, (size_t)unit);
    a.cols_per_split = pl.cols_per_split;
    a.splits = pl.splits;
    a.n_rb = pl.n_rb;
    a.n_hi = pl.n_rb;
    a.cps_lo = pl.cols_per_split;
    a.part_ld = pl.n_rb * RB;
    a.counters = counters;
}

// The exact one-wave plan (fill_plan, cov_internal.h) in this kernel's tiles.
static void fill_segment(PairArgs& a, int n_cols, int budget, int unit) { fill_plan(a, n_cols, budget, unit, kTile / unit); }

static int seg_ctas(const PairArgs& a) { return a.n_hi * a.splits + (a.n_rb - a.n_hi) * (a.splits - 1); }

// Plans and launches one or two all-pairs passes of one kernel family in a
// single grid.  seg[k] covers seg[k].n_rows rows x n_cols[k] columns; with
// two segments the CTA slots are shared in proportion to their pair counts
// and seg[1]'s partials follow seg[0]'s in the partial buffer.
static cov_status run_pairs(cov_ctx* ctx, int d, int family, PairArgs* seg, const int* n_cols, int nseg,
                            const int* cnt_off, unsigned* counters, cudaStream_t st) {
    // Fixed-offset updates of every segment with records: exponents on the
    // tensor cores (128-row CTAs, 128-column tiles)
    bool tc = family == M_GO && ctx->use_tc && d <= 3;
    for (int k = 0; k < nseg; ++k) tc = tc && seg[k].fixed && seg[k].rec0 && seg[k].rech;
    // the weighted (barycentre) passes may take another row count per thread (build flag)
    const bool weighted = family == M_WY || family == M_WX || family == M_GW;
    const int R = effective_R(d, (weighted && COV_BARY_R > 0) ? COV_BARY_R : ctx->rows_per_thread);
    const int RB = tc ? kTcRows : 32 * R;
    const int unit = tc ? kTcCols : 8;
    const int fixed_cost = tc ? 2 * kTcCols : 64;
    // one wave: as many CTAs as can be resident (the register budget, and
    // for the tensor-core kernel its tensor memory, decides how many per SM),
    // capped by the tuning option
    int occ = 1;
    if (tc)
        launch_tc_d(d, PairLaunch{}, 0, st, &occ);
    else
        launch_pairs_d(d, R, family, PairLaunch{}, 0, st, &occ);
    // inside a batch many problems' launches share the GPU: plan each for its share of the slots
    const int slots_all = std::max(1, std::min(ctx->num_sms * std::min(occ, ctx->ctas_per_sm), kMaxSlots));
    const int slots = ctx->plan_share >= 100 ? slots_all : std::max(1, slots_all * ctx->plan_share / 100);
    const int nacc = family == M_SVGD ? d : ((family == M_WY || family == M_WX || family == M_GW) ? 2 + d : 2);
    // uniform plan; when it is one wave that already fills at least half the
    // slots, re-plan to fill them exactly (CUDA-core kernel)
    // The tensor-core kernel holds one CTA per SM, so row blocks alone often
    // end in a part-filled last wave (512 row blocks on 148 SMs: 3.46 waves);
    // its split search reaches up to 8 waves to square them off, within the
    // partial-buffer bound (splits x row blocks x RB <= waves x slots x RB +
    // the rows, against kPartRows)
    const int max_waves = tc ? (int)std::min<long long>(8, 2LL * kMaxSlots * 256 / ((long long)slots * RB)) : 2;
    auto plan = [&](PairArgs& a, int nc, int budget, unsigned* cnt) {
        plan_segment(a, nc, RB, budget, cnt, unit, fixed_cost, std::max(2, max_waves));
        const long long ctas = (long long)a.n_rb * a.splits;
        if (!tc && ctas <= budget && 2 * ctas >= budget && budget > a.n_rb) fill_segment(a, nc, budget, unit);
    };
    PairLaunch L{};
    if (nseg == 1) {
        plan(seg[0], n_cols[0], slots, counters + cnt_off[0]);
        L.seg[0] = seg[0];
        L.seg[1] = seg[0];
        L.ctas0 = seg_ctas(seg[0]);
    } else {
        const double w0 = (double)seg[0].n_rows * n_cols[0], w1 = (double)seg[1].n_rows * n_cols[1];
        int s0 = (int)llround(slots * w0 / (w0 + w1));
        s0 = std::max(1, std::min(s0, slots - 1));
        const int s1 = std::max(1, slots - s0);
        plan(seg[0], n_cols[0], s0, counters + cnt_off[0]);
        plan(seg[1], n_cols[1], s1, counters + cnt_off[1]);
        seg[1].part = seg[0].part + (size_t)nacc * seg[0].splits * seg[0].part_ld;
        L.seg[0] = seg[0];
        L.seg[1] = seg[1];
        L.ctas0 = seg_ctas(seg[0]);
    }
    const int total = L.ctas0 + (nseg == 2 ? seg_ctas(seg[1]) : 0);
    const cudaError_t e = tc ? launch_tc_d(d, L, total, st, nullptr) : launch_pairs_d(d, R, family, L, total, st, nullptr);
    return cuda_failed(ctx, e) ? COV_ERR_CUDA : COV_OK;
}

// with_part = false leaves part/counters to the caller (a recorded forward
// keeps many tapes and shares one split buffer between them).
static SkBufs carve_sinkhorn(Carver& cv, int T, int M, int d, bool with_part = true, bool with_rec = false) {
    SkBufs B{};
    B.Tp = (int)round_up((size_t)T, kRowPad);
    B.Mp = (int)round_up((size_t)M, kRowPad);
    B.xs = cv.take<float>((size_t)d * B.Tp);
    B.ys = cv.take<float>((size_t)d * B.Mp);
    B.hx = cv.take<float>(B.Tp);
    B.hy = cv.take<float>(B.Mp);
    B.hp0 = cv.take<float>(B.Tp);
    B.hp1 = cv.take<float>(B.Tp);
    B.lb = cv.take<float>(B.Mp);
    B.nx = cv.take<float>(B.Tp);
    B.ny = cv.take<float>(B.Mp);
    B.bary = cv.take<float>((size_t)d * B.Tp);
    B.scal = cv.take<float>(16);
    B.cnt_ld = cnt_ld_for(B.Tp, B.Mp);
    B.part_floats = (size_t)(2 + d) * (kPartRows + B.Tp + B.Mp);
    if (with_part) {
        B.counters = cv.take<unsigned>((size_t)M_COUNT * B.cnt_ld);
        B.part = cv.take<float>(B.part_floats);
    }
    if (with_rec && d <= 3) {
        B.c0x = cv.take<float>((size_t)kTcRecC * B.Tp);
        B.c0y = cv.take<float>((size_t)kTcRecC * B.Mp);
        B.hrx = cv.take<float>((size_t)kTcRecH * B.Tp);
        B.hrp0 = cv.take<float>((size_t)kTcRecH * B.Tp);
        B.hrp1 = cv.take<float>((size_t)kTcRecH * B.Tp);
        B.hry = cv.take<float>((size_t)kTcRecH * B.Mp);
    }
    return B;
}

size_t sinkhorn_split_bytes(int T, int M, int d) {
    const size_t Tp = round_up((size_t)T, kRowPad), Mp = round_up((size_t)M, kRowPad);
    Carver cv(nullptr);
    cv.take<unsigned>((size_t)M_COUNT * cnt_ld_for((int)Tp, (int)Mp));
    cv.take<float>((size_t)(2 + d) * (kPartRows + Tp + Mp));
    return round_up(cv.off, 256);
}

void sinkhorn_reference_stats(const float* y, int M, int d, const float* b, float* scal, cudaStream_t stream) {
    launch_pdl(sk_centre_kernel, dim3(1), dim3(kCentreThreads), 0, stream, y, M, d, b, scal);
}

size_t sinkhorn_ws_bytes(int T, int M, int d) {
    Carver cv(nullptr);
    carve_sinkhorn(cv, T, M, d, true, true);
    return round_up(cv.off, 256);
}

cov_status sinkhorn_field_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int x_ld, int T,
                             const float* y, const float* b, int M, int d, float eps, int n_iter, int flags,
                             float* f, float* g, float* p, float* a_out, cudaStream_t stream,
                             const float* scal_given, float eps_start, float eps_decay) {
    if (!ctx || !x || !y || T < 1 || M < 1 || d < 1 || d > COV_MAX_D || x_ld < d || n_iter < 0 ||
        !(eps > 0.f) || !isfinite(eps))
        return COV_ERR_INVALID_ARG;
    const bool scaled = eps_start > eps;
    if (scaled && (!isfinite(eps_start) || !(eps_decay > 0.f) || !(eps_decay < 1.f))) return COV_ERR_INVALID_ARG;
    const int warm = (flags & COV_WARM_START) ? 1 : 0;
    if (warm && (!f || !g || !p)) return COV_ERR_INVALID_ARG;
    Carver cv(ws);
    SkBufs B = carve_sinkhorn(cv, T, M, d, true, true);
    if (!ws || cv.off > ws_bytes) return COV_ERR_WORKSPACE;
    if (cuda_failed(ctx, cudaMemsetAsync(B.counters, 0, sizeof(unsigned) * M_COUNT * B.cnt_ld, stream)))
        return COV_ERR_CUDA;

    // stage eps: the first iteration's (eps-scaling), else eps throughout
    double eps_cur = scaled ? anneal_eps(eps, eps_start, eps_decay, 0) : (double)eps;
    const double epsln2_0 = eps_cur * 0.69314718055994531;
    const double epsln2 = (double)eps * 0.69314718055994531;
    const float sigma = (float)sqrt(epsln2);
    const float log2a = (float)(-log2((double)T));
    if (scal_given)
        B.scal = const_cast<float*>(scal_given);
    else
        launch_pdl(sk_centre_kernel, dim3(1), dim3(kCentreThreads), 0, stream, y, M, d, b, B.scal);
    const int np = std::max(B.Tp, B.Mp);
    launch_pdl(sk_prep_kernel, dim3((np + 255) / 256), dim3(256), 0, stream, x, x_ld, T, y, M, b, d, (float)(1.0 / sqrt(epsln2_0)),
                                                         (float)(1.0 / epsln2_0), log2a, warm, f, g, p, B,
                                                         ctx->status);
    PairArgs base{};
    base.status = ctx->status;
    base.spin_limit = ctx->spin_limit;
    base.log2a = log2a;
    base.part = B.part;
    base.pre_ok = 1;
    float* hp_cur = B.hp0;
    float* hp_nxt = B.hp1;
    float* hrp_cur = B.hrp0;  // h records of hp_cur / hp_nxt (tensor-core path)
    float* hrp_nxt = B.hrp1;
    bool first = true;  // the first pass reads what the prep kernel just wrote
    cov_status r = COV_OK;
    // the tensor-core records of the current state (after the prep or a
    // rescale; every update's epilogue then keeps its rows' h records current)
    // records are kept only when the tensor-core path will run: always with
    // the option at 1; with it at 2 when both launches of an iteration
    // (g + p: M T + T^2 pairs, f: T M pairs) are of at least 2^30 pairs
    const long long pairs_min = std::min((long long)M * T + (long long)T * T, (long long)T * M);
    const bool want_tc = ctx->use_tc == 1 || (ctx->use_tc == 2 && pairs_min >= kTcAutoPairs);
    const bool recs = B.c0x != nullptr && want_tc;
    auto build_records = [&]() {
        if (!recs) return;
        const int nb = (np + 255) / 256;
        if (d == 1)
            launch_pdl(tc_records_kernel<1>, dim3(nb), dim3(256), 0, stream, B.xs, B.Tp, B.ys, B.Mp, B.hx, hp_cur, hp_nxt, B.hy, B.c0x,
                                                         B.c0y, B.hrx, hrp_cur, hrp_nxt, B.hry);
        else if (d == 2)
            launch_pdl(tc_records_kernel<2>, dim3(nb), dim3(256), 0, stream, B.xs, B.Tp, B.ys, B.Mp, B.hx, hp_cur, hp_nxt, B.hy, B.c0x,
                                                         B.c0y, B.hrx, hrp_cur, hrp_nxt, B.hry);
        else
            launch_pdl(tc_records_kernel<3>, dim3(nb), dim3(256), 0, stream, B.xs, B.Tp, B.ys, B.Mp, B.hx, hp_cur, hp_nxt, B.hy, B.c0x,
                                                         B.c0y, B.hrx, hrp_cur, hrp_nxt, B.hry);
        first = true;
    };
    build_records();
    // move the state to another eps (coordinates and potential terms), on
    // the stream before the next pass; that pass then waits for it
    auto to_eps = [&](double e_new) {
        if (e_new == eps_cur) return;
        const int nb = (np + 255) / 256;
        launch_pdl(sk_rescale_kernel, dim3(nb), dim3(256), 0, stream, B, T, M, d, (float)sqrt(eps_cur / e_new), (float)(eps_cur / e_new),
                                                  log2a, hp_cur, ctx->status);
        eps_cur = e_new;
        first = true;
        build_records();
    };
    int stable = 0;            // iterations run at the current eps
    bool warm_origin = warm;   // the warm-start potentials are still at the current eps
    bool bary_done = false;    // the last f-update already formed the cross barycentre
    for (int it = 0; it < n_iter && r == COV_OK; ++it) {
        if (scaled) {
            const double e_it = anneal_eps(eps, eps_start, eps_decay, it);
            if (e_it != eps_cur) {
                stable = 0;
                warm_origin = false;
            }
            to_eps(e_it);
        }
        // The updates run with a fixed row offset (M_GO) from the second
        // iteration at one eps on, or at once from warm-start potentials: the
        // previous log-sum-exp of the row, read back from the potentials it
        // produced (g: lb - hy, f: log2 a - hx, p: log2 a + hp^(t-2) -
        // 2 hp^(t-1), hp^(t-2) being the values the first update at this eps
        // started from); before the first p-update of a warm start, the fixed
        // point of that update, log2 a - hp (exact at convergence).  From a
        // cold start the row log-sum-exps of the benchmark workloads move by
        // under 2 bits from the first iteration to the second (FP64 oracle,
        // eps = 0.005 and 0.002), far inside the guards' 2^-60 .. 2^100.
        const bool fixed = stable >= 1 || warm_origin;
        const bool p_prev = stable >= 1;
        const int fam = fixed ? M_GO : M_G;
        // launch A: g-update (rows y, columns x) and self p-update (rows x,
        // columns x) -- independent, same column set
        PairArgs sg[2] = {base, base};
        sg[0].rows = B.ys; sg[0].row_ld = B.Mp; sg[0].n_rows = M;
        sg[0].cols = B.xs; sg[0].colh = B.hx; sg[0].col_ld = B.Tp;
        sg[0].out_h = B.hy; sg[0].in_h = B.lb; sg[0].emode = M_G;
        sg[0].oa = B.lb; sg[0].oca = 1.f; sg[0].ob = B.hy; sg[0].ocb = -1.f; sg[0].oc0 = 0.f;  // lb - hy
        sg[0].fixed = fixed;
        if (recs) { sg[0].rec0 = B.c0x; sg[0].rech = B.hrx; sg[0].out_rec = B.hry; }
        sg[1].rows = B.xs; sg[1].row_ld = B.Tp; sg[1].n_rows = T;
        sg[1].cols = B.xs; sg[1].colh = hp_cur; sg[1].col_ld = B.Tp;
        sg[1].out_h = hp_nxt; sg[1].in_h = hp_cur; sg[1].emode = M_P;
        if (p_prev) {  // log2 a + hp^{t-2} - 2 hp^{t-1} (hp_nxt still holds hp^{t-2})
            sg[1].oa = hp_nxt; sg[1].oca = 1.f; sg[1].ob = hp_cur; sg[1].ocb = -2.f; sg[1].oc0 = log2a;
        } else {       // log2 a - hp^{t-1}
            sg[1].oa = hp_cur; sg[1].oca = -1.f; sg[1].ob = nullptr; sg[1].ocb = 0.f; sg[1].oc0 = log2a;
        }
        sg[1].fixed = fixed;
        if (recs) { sg[1].rec0 = B.c0x; sg[1].rech = hrp_cur; sg[1].out_rec = hrp_nxt; }
        if (first) sg[0].pre_ok = sg[1].pre_ok = 0;
        first = false;
        const int ncA[2] = {T, T}, coA[2] = {M_G * B.cnt_ld, M_P * B.cnt_ld};
        r = run_pairs(ctx, d, fam, sg, ncA, 2, coA, B.counters, stream);
        if (r != COV_OK) break;
        // launch B: f-update (rows x, columns y)
        PairArgs a = base;
        a.rows = B.xs; a.row_ld = B.Tp; a.n_rows = T;
        a.cols = B.ys; a.colh = B.hy; a.col_ld = B.Mp;
        a.out_h = B.hx; a.emode = M_F;
        a.oa = B.hx; a.oca = -1.f; a.ob = nullptr; a.oc0 = log2a;  // log2 a - hx
        a.fixed = fixed;
        if (recs) { a.rec0 = B.c0y; a.rech = B.hry; a.out_rec = B.hrx; }
        // the last f-update, at the target eps on the CUDA cores, also forms
        // the cross barycentre of its own softmax (the gradient pass's first
        // half reads the same columns and the same final g, and normalises by
        // its own sum): one pass fewer
        const bool with_bary = a_out && it == n_iter - 1 && !recs && eps_cur == (double)eps;
        if (with_bary) a.bary = B.bary;
        const int ncB[1] = {M}, coB[1] = {(with_bary ? M_GW : M_F) * B.cnt_ld};
        r = run_pairs(ctx, d, with_bary ? M_GW : fam, &a, ncB, 1, coB, B.counters, stream);
        bary_done = with_bary;
        std::swap(hp_cur, hp_nxt);
        std::swap(hrp_cur, hrp_nxt);
        ++stable;
    }
    if (r != COV_OK) return r;
    to_eps((double)eps);  // the field and the returned potentials are at the target eps
    if (a_out) {
        if (!bary_done) {
            PairArgs a = base;  // cross barycentre: (sum_j pi_ij yhat_j) - xhat_i
            a.rows = B.xs; a.row_ld = B.Tp; a.n_rows = T;
            a.cols = B.ys; a.colh = B.hy; a.col_ld = B.Mp;
            a.bary = B.bary;
            if (first) a.pre_ok = 0;
            first = false;
            const int nc1[1] = {M}, co1[1] = {M_WY * B.cnt_ld};
            r = run_pairs(ctx, d, M_WY, &a, nc1, 1, co1, B.counters, stream);
            if (r != COV_OK) return r;
        }
        PairArgs a = base;  // self barycentre and the field 2 sigma (ybar - xbar)
        a.rows = B.xs; a.row_ld = B.Tp; a.n_rows = T;
        a.cols = B.xs; a.colh = hp_cur; a.col_ld = B.Tp;
        a.bary = B.bary; a.a_out = a_out; a.a_scale = 2.0f * sigma;
        if (first) a.pre_ok = 0;
        first = false;
        const int nc2[1] = {T}, co2[1] = {M_WX * B.cnt_ld};
        r = run_pairs(ctx, d, M_WX, &a, nc2, 1, co2, B.counters, stream);
        if (r != COV_OK) return r;
    }
    if (f || g || p) {
        const int nf = std::max(T, M);
        launch_pdl(sk_finish_kernel, dim3((nf + 255) / 256), dim3(256), 0, stream, T, M, (float)epsln2, log2a, B, hp_cur, f, g, p,
                                                               ctx->status);
    }
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

// ---------------------------------------------------------------------------
// Recorded forward for the adjoint: the same iterations as sinkhorn_field_ws
// (cold start), every iteration's per-column terms kept in their own slot,
// plus the barycentric offsets of each update's softmax and one further
// self update whose log-sum-exp normalises the self term of the field.
// ---------------------------------------------------------------------------
__global__ void tape_pad_kernel(SkTape tp) {
    pdl_prologue();
    // padding entries of every history slot: hx (n+1 slots) and hp (n+2
    // slots) over [T, Tp), hy (n+1 slots) over [M, Mp)
    const int n = tp.n_iter;
    const int padx = tp.Tp - tp.T, pady = tp.Mp - tp.M;
    const long long nx = padx > 0 ? (long long)(2 * n + 3) * padx : 0;
    const long long ny = pady > 0 ? (long long)(n + 1) * pady : 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nx + ny;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < nx) {
            const long long slot = e / padx, i = tp.T + e % padx;
            if (slot <= n) tp.hx[slot * tp.Tp + i] = kPadH;
            else tp.hp[(slot - n - 1) * tp.Tp + i] = kPadH;
        } else {
            const long long f = e - nx, slot = f / pady, j = tp.M + f % pady;
            tp.hy[slot * tp.Mp + j] = kPadH;
        }
    }
}

static void carve_tape(Carver& cv, int n_iter, int d, int Tp, int Mp, SkTape* tp) {
    tp->hx = cv.take<float>((size_t)(n_iter + 1) * Tp);
    tp->hy = cv.take<float>((size_t)(n_iter + 1) * Mp);
    tp->hp = cv.take<float>((size_t)(n_iter + 2) * Tp);
    tp->Df = cv.take<float>((size_t)(n_iter + 1) * d * Tp);
    tp->Dg = cv.take<float>((size_t)(n_iter + 1) * d * Mp);
    tp->Dp = cv.take<float>((size_t)(n_iter + 1) * d * Tp);
}

size_t sinkhorn_tape_bytes(int T, int M, int d, int n_iter, bool with_part) {
    Carver cv(nullptr);
    SkBufs B = carve_sinkhorn(cv, T, M, d, with_part);
    SkTape tp{};
    carve_tape(cv, n_iter, d, B.Tp, B.Mp, &tp);
    return round_up(cv.off, 256);
}

cov_status sinkhorn_tape_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int x_ld, int T,
                            const float* y, const float* b, int M, int d, float eps, int n_iter,
                            const float* scal_given, SkTape* tape, size_t* used, cudaStream_t stream,
                            float* split_ws, float* a_out) {
    if (!ctx || !x || !y || !tape || T < 1 || M < 1 || d < 1 || d > COV_MAX_D || x_ld < d || n_iter < 0 ||
        !(eps > 0.f) || !isfinite(eps))
        return COV_ERR_INVALID_ARG;
    Carver cv(ws);
    SkBufs B = carve_sinkhorn(cv, T, M, d, split_ws == nullptr);
    if (split_ws) {
        Carver cs(split_ws);
        B.counters = cs.take<unsigned>((size_t)M_COUNT * B.cnt_ld);
        B.part = cs.take<float>(B.part_floats);
    }
    SkTape tp{};
    carve_tape(cv, n_iter, d, B.Tp, B.Mp, &tp);
    if (!ws || cv.off > ws_bytes) return COV_ERR_WORKSPACE;
    if (used) *used = round_up(cv.off, 256);
    const int n = n_iter;
    const double epsln2 = (double)eps * 0.69314718055994531;
    tp.n_iter = n;
    tp.T = T; tp.M = M; tp.d = d; tp.Tp = B.Tp; tp.Mp = B.Mp;
    tp.eps = eps;
    tp.sigma = (float)sqrt(epsln2);
    tp.log2a = (float)(-log2((double)T));
    tp.xs = B.xs; tp.ys = B.ys; tp.lb = B.lb;
    // slot 0 of each history is the cold start written by the prep kernel
    B.hx = tp.hx;
    B.hy = tp.hy;
    B.hp0 = tp.hp;
    if (cuda_failed(ctx, cudaMemsetAsync(B.counters, 0, sizeof(unsigned) * M_COUNT * B.cnt_ld, stream)))
        return COV_ERR_CUDA;
    if (scal_given)
        B.scal = const_cast<float*>(scal_given);
    else
        launch_pdl(sk_centre_kernel, dim3(1), dim3(kCentreThreads), 0, stream, y, M, d, b, B.scal);
    const int np = std::max(B.Tp, B.Mp);
    launch_pdl(sk_prep_kernel, dim3((np + 255) / 256), dim3(256), 0, stream, x, x_ld, T, y, M, b, d, (float)(1.0 / tp.sigma),
                                                         (float)(1.0 / epsln2), tp.log2a, 0, nullptr, nullptr,
                                                         nullptr, B, ctx->status);
    launch_pdl(tape_pad_kernel, dim3(std::min(1024, (int)((2LL * n + 2) * B.Tp / 256 + 1))), dim3(256), 0, stream, tp);
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    PairArgs base{};
    base.status = ctx->status;
    base.spin_limit = ctx->spin_limit;
    base.log2a = tp.log2a;
    base.part = B.part;
    base.pre_ok = 1;
    bool first = true;
    cov_status r = COV_OK;
    for (int t = 1; t <= n && r == COV_OK; ++t) {
        float* hx_prev = tp.hx + (size_t)(t - 1) * B.Tp;
        float* hx_t = tp.hx + (size_t)t * B.Tp;
        float* hy_t = tp.hy + (size_t)t * B.Mp;
        float* hp_prev = tp.hp + (size_t)(t - 1) * B.Tp;
        float* hp_t = tp.hp + (size_t)t * B.Tp;
        PairArgs sg[2] = {base, base};
        sg[0].rows = B.ys; sg[0].row_ld = B.Mp; sg[0].n_rows = M;
        sg[0].cols = B.xs; sg[0].colh = hx_prev; sg[0].col_ld = B.Tp;
        sg[0].out_h = hy_t; sg[0].in_h = B.lb; sg[0].emode = M_G;
        sg[0].bary = tp.Dg + (size_t)t * d * B.Mp;
        sg[1].rows = B.xs; sg[1].row_ld = B.Tp; sg[1].n_rows = T;
        sg[1].cols = B.xs; sg[1].colh = hp_prev; sg[1].col_ld = B.Tp;
        sg[1].out_h = hp_t; sg[1].in_h = hp_prev; sg[1].emode = M_P;
        sg[1].bary = tp.Dp + (size_t)t * d * B.Tp;
        if (first) sg[0].pre_ok = sg[1].pre_ok = 0;
        first = false;
        const int ncA[2] = {T, T}, coA[2] = {M_G * B.cnt_ld, M_P * B.cnt_ld};
        r = run_pairs(ctx, d, M_GW, sg, ncA, 2, coA, B.counters, stream);
        if (r != COV_OK) break;
        PairArgs a = base;
        a.rows = B.xs; a.row_ld = B.Tp; a.n_rows = T;
        a.cols = B.ys; a.colh = hy_t; a.col_ld = B.Mp;
        a.out_h = hx_t; a.emode = M_F;
        a.bary = tp.Df + (size_t)t * d * B.Tp;
        const int ncB[1] = {M}, coB[1] = {M_F * B.cnt_ld};
        r = run_pairs(ctx, d, M_GW, &a, ncB, 1, coB, B.counters, stream);
    }
    if (r != COV_OK) return r;
    // the cross normaliser of the field: f-update on the last g (only needed
    // when no iteration ran; otherwise it is hx^n itself)
    if (n == 0) {
        PairArgs a = base;
        a.rows = B.xs; a.row_ld = B.Tp; a.n_rows = T;
        a.cols = B.ys; a.colh = tp.hy; a.col_ld = B.Mp;
        a.out_h = tp.hx; a.emode = M_F;
        if (first) a.pre_ok = 0;
        first = false;
        const int nc[1] = {M}, co[1] = {M_F * B.cnt_ld};
        r = run_pairs(ctx, d, M_G, &a, nc, 1, co, B.counters, stream);
        if (r != COV_OK) return r;
    }
    {   // one more self update: hp^{n+1}, the normaliser of the self softmax
        PairArgs a = base;
        a.rows = B.xs; a.row_ld = B.Tp; a.n_rows = T;
        a.cols = B.xs; a.colh = tp.hp + (size_t)n * B.Tp; a.col_ld = B.Tp;
        a.out_h = tp.hp + (size_t)(n + 1) * B.Tp; a.in_h = a.colh; a.emode = M_P;
        if (first) a.pre_ok = 0;
        first = false;
        const int nc[1] = {T}, co[1] = {M_P * B.cnt_ld};
        r = run_pairs(ctx, d, M_G, &a, nc, 1, co, B.counters, stream);
        if (r != COV_OK) return r;
    }
    if (a_out) {  // the field itself (Eq. 7) from the last potentials, as sinkhorn_field_ws
        PairArgs a = base;
        a.rows = B.xs; a.row_ld = B.Tp; a.n_rows = T;
        a.cols = B.ys; a.colh = tp.hy + (size_t)n * B.Mp; a.col_ld = B.Mp;
        a.bary = B.bary;
        const int nc1[1] = {M}, co1[1] = {M_WY * B.cnt_ld};
        r = run_pairs(ctx, d, M_WY, &a, nc1, 1, co1, B.counters, stream);
        if (r != COV_OK) return r;
        a = base;
        a.rows = B.xs; a.row_ld = B.Tp; a.n_rows = T;
        a.cols = B.xs; a.colh = tp.hp + (size_t)n * B.Tp; a.col_ld = B.Tp;
        a.bary = B.bary; a.a_out = a_out; a.a_scale = 2.0f * tp.sigma;
        const int nc2[1] = {T}, co2[1] = {M_WX * B.cnt_ld};
        r = run_pairs(ctx, d, M_WX, &a, nc2, 1, co2, B.counters, stream);
        if (r != COV_OK) return r;
    }
    tp.scal = B.scal;
    *tape = tp;
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

// ---------------------------------------------------------------------------
// Stein variational field and the mixture score
// ---------------------------------------------------------------------------
}  // namespace cov

cov_status cov::make_gmm_params(const cov_gmm* g, int d, GmmParams* out) {
    if (!g || !out || g->K < 1 || g->K > COV_MAX_GMM || g->d != d || !g->w || !g->mu || !g->sigma)
        return COV_ERR_INVALID_ARG;
    double wsum = 0.0;
    for (int k = 0; k < g->K; ++k) {
        if (!(g->w[k] > 0.f) || !(g->sigma[k] > 0.f) || !isfinite(g->w[k]) || !isfinite(g->sigma[k]))
            return COV_ERR_INVALID_ARG;
        wsum += g->w[k];
    }
    GmmParams P{};
    P.K = g->K;
    P.d = d;
    for (int k = 0; k < g->K; ++k) {
        const double s = g->sigma[k];
        P.lw[k] = (float)(log2(g->w[k] / wsum) - d * log2(s));
        P.inv2s2[k] = (float)(1.0 / (2.0 * s * s * 0.69314718055994531));
        P.invs2[k] = (float)(1.0 / (s * s));
        for (int c = 0; c < d; ++c) {
            if (!isfinite(g->mu[k * d + c])) return COV_ERR_INVALID_ARG;
            P.mu[k * COV_MAX_D + c] = g->mu[k * d + c];
        }
    }
    *out = P;
    return COV_OK;
}

namespace cov {

// grad log q(x) for the mixture: softmax responsibilities in base 2.
__device__ __forceinline__ void gmm_score_at(const GmmParams& G, const float* xv, int d, float* sc) {
    float t[COV_MAX_GMM];
    float tm = kNegBig;
    for (int k = 0; k < G.K; ++k) {
        float r2 = 0.f;
        for (int c = 0; c < d; ++c) {
            const float dv = xv[c] - G.mu[k * COV_MAX_D + c];
            r2 = fmaf(dv, dv, r2);
        }
        t[k] = G.lw[k] - r2 * G.inv2s2[k];
        tm = fmaxf(tm, t[k]);
    }
    float den = 0.f;
    for (int c = 0; c < d; ++c) sc[c] = 0.f;
    for (int k = 0; k < G.K; ++k) {
        const float e = ex2(t[k] - tm);
        den += e;
        for (int c = 0; c < d; ++c) sc[c] = fmaf(e * G.invs2[k], G.mu[k * COV_MAX_D + c] - xv[c], sc[c]);
    }
    const float inv = 1.0f / den;
    for (int c = 0; c < d; ++c) sc[c] *= inv;
}

__global__ void gmm_score_kernel(const float* __restrict__ x, int T, int d, GmmParams G, float* __restrict__ out,
                                 unsigned* status) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    float xv[COV_MAX_D], sc[COV_MAX_D];
    for (int c = 0; c < d; ++c) xv[c] = x[(size_t)i * d + c];
    gmm_score_at(G, xv, d, sc);
    bool ok = true;
    for (int c = 0; c < d; ++c) {
        out[(size_t)i * d + c] = sc[c];
        ok &= finitef(sc[c]);
    }
    if (!ok) raise_status(status, kDevNonfinite);
}

// Score of a pixel-density reference (d = 2): q is the bilinear interpolant
// of map[iy][ix] with pixel centres at ((ix + 1/2)/W, (iy + 1/2)/H), each
// coordinate clamped to the outermost centres (constant extension, zero
// gradient outside), score = grad q / q.  One thread per point; the map
// (1 MB at 512^2) stays in L2.
__device__ __forceinline__ void density_score_at(const float* __restrict__ map, int H, int W, float x0, float x1,
                                                 float* sc) {
    float u = fmaf(x0, (float)W, -0.5f), v = fmaf(x1, (float)H, -0.5f);
    const bool inx = u > 0.f && u < (float)(W - 1), iny = v > 0.f && v < (float)(H - 1);
    u = fminf(fmaxf(u, 0.f), (float)(W - 1));
    v = fminf(fmaxf(v, 0.f), (float)(H - 1));
    const int ix = min((int)floorf(u), W - 2), iy = min((int)floorf(v), H - 2);
    const float fx = u - (float)ix, fy = v - (float)iy;
    const float q00 = __ldg(map + (size_t)iy * W + ix), q10 = __ldg(map + (size_t)iy * W + ix + 1);
    const float q01 = __ldg(map + (size_t)(iy + 1) * W + ix), q11 = __ldg(map + (size_t)(iy + 1) * W + ix + 1);
    const float q0 = fmaf(fx, q10 - q00, q00), q1 = fmaf(fx, q11 - q01, q01);
    const float q = fmaf(fy, q1 - q0, q0);
    const float gx = inx ? (float)W * fmaf(fy, (q11 - q01) - (q10 - q00), q10 - q00) : 0.f;
    const float gy = iny ? (float)H * (q1 - q0) : 0.f;
    const float iq = 1.0f / q;
    sc[0] = gx * iq;
    sc[1] = gy * iq;
}

__global__ void density_score_kernel(const float* __restrict__ map, int H, int W, const float* __restrict__ x,
                                     int x_ld, int T, float* __restrict__ score, unsigned* status) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    float sc[2];
    density_score_at(map, H, W, x[(size_t)i * x_ld], x[(size_t)i * x_ld + 1], sc);
    score[(size_t)i * 2] = sc[0];
    score[(size_t)i * 2 + 1] = sc[1];
    if (!(finitef(sc[0]) && finitef(sc[1]))) raise_status(status, kDevNonfinite);
}

cov_status density_score_launch(cov_ctx* ctx, const float* map, int H, int W, const float* x, int x_ld, int T,
                                float* score, cudaStream_t stream) {
    if (!ctx || !map || !x || !score || T < 1 || H < 2 || W < 2 || x_ld < 2) return COV_ERR_INVALID_ARG;
    launch_pdl(density_score_kernel, dim3((T + 255) / 256), dim3(256), 0, stream, map, H, W, x, x_ld, T, score, ctx->status);
    return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;
}

// xt = x / (h sqrt(2 ln 2)),  st = score h / sqrt(2 ln 2); padding: xt far away, st = 0.
__global__ void svgd_prep_kernel(const float* __restrict__ x, int x_ld, int T, int d, int Tp,
                                 const float* __restrict__ score, GmmParams G, int use_gmm, float inv_hs, float hs,
                                 float* __restrict__ xt, float* __restrict__ st, unsigned* status) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Tp) return;
    if (i >= T) {
        for (int c = 0; c < d; ++c) {
            xt[(size_t)c * Tp + i] = kSvgdPad;
            st[(size_t)c * Tp + i] = 0.f;
        }
        return;
    }
    float xv[COV_MAX_D], sc[COV_MAX_D];
    for (int c = 0; c < d; ++c) xv[c] = x[(size_t)i * x_ld + c];
    if (use_gmm) {
        gmm_score_at(G, xv, d, sc);
    } else {
        for (int c = 0; c < d; ++c) sc[c] = score[(size_t)i * d + c];
    }
    bool ok = true;
    for (int c = 0; c < d; ++c) {
        xt[(size_t)c * Tp + i] = xv[c] * inv_hs;
        st[(size_t)c * Tp + i] = sc[c] * hs;
        ok &= finitef(xv[c]) && finitef(sc[c]);
    }
    if (!ok) raise_status(status, kDevNonfinite);
}

// Stein field of a short trajectory in one launch (T <= kSvSmallMaxT):
// every CTA forms the prescaled coordinates and scores of all T points in
// shared memory (the mixture score recomputed per CTA, T K exponentials,
// small next to its rows' pairs), then sums its 32 rows over all T columns
// in the arithmetic of the all-pairs kernel's Stein pass,
//   a_i = a_scale sum_j 2^(-|xt_i - xt_j|^2) (st_j + xt_i - xt_j),
// warp q taking the columns j = q (mod 8) for all 32 rows (its lanes read the
// same column: shared-memory broadcasts), and the 8 partial sums of a row
// added in warp order.  The points are read as x[j x_ld + c] for j < T
// (float coordinates, or the FP64 states of a solve, which this also
// extracts).
constexpr int kSvSmallRows = 32;
constexpr int kSvSmallSplits = 8;
constexpr int kSvSmallThreads = kSvSmallRows * kSvSmallSplits;
constexpr int kSvSmallMaxT = 1024;

template <int D, typename XT>
__global__ void __launch_bounds__(kSvSmallThreads) svgd_small_kernel(const XT* __restrict__ x, int x_ld, int T,
                                                                     const float* __restrict__ score, GmmParams G,
                                                                     int use_gmm, float inv_hs, float hs,
                                                                     float a_scale, float* __restrict__ a_out,
                                                                     unsigned* status) {
    pdl_prologue();
    extern __shared__ float sv[];  // xt [D][T], st [D][T]
    __shared__ float red[kSvSmallSplits][D][kSvSmallRows];
    float* xs = sv;
    float* ss = sv + (size_t)D * T;
    bool ok = true;
    for (int j = threadIdx.x; j < T; j += kSvSmallThreads) {
        float xv[D], sc[D];
#pragma unroll
        for (int c = 0; c < D; ++c) xv[c] = (float)x[(size_t)j * x_ld + c];
        if (use_gmm) {
            gmm_score_at(G, xv, D, sc);
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) sc[c] = score[(size_t)j * D + c];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            xs[(size_t)c * T + j] = xv[c] * inv_hs;
            ss[(size_t)c * T + j] = sc[c] * hs;
            ok &= finitef(xv[c]) && finitef(sc[c]);
        }
    }
    if (!ok && blockIdx.x == 0) raise_status(status, kDevNonfinite);
    __syncthreads();
    const int r = threadIdx.x % kSvSmallRows, q = threadIdx.x / kSvSmallRows;
    const int i = min(blockIdx.x * kSvSmallRows + r, T - 1);  // rows past T repeat the last (not stored)
    float xi[D], acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        xi[c] = xs[(size_t)c * T + i];
        acc[c] = 0.f;
    }
    for (int j = q; j < T; j += kSvSmallSplits) {
        float dl[D], r2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            dl[c] = xi[c] - xs[(size_t)c * T + j];
            r2 = fmaf(dl[c], dl[c], r2);
        }
        const float k = ex2(-r2);
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = fmaf(k, ss[(size_t)c * T + j] + dl[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) red[q][c][r] = acc[c];
    __syncthreads();
    if (threadIdx.x < kSvSmallRows * D) {
        const int rr = threadIdx.x % kSvSmallRows, c = threadIdx.x / kSvSmallRows;
        const int ii = blockIdx.x * kSvSmallRows + rr;
        float sum = 0.f;
#pragma unroll
        for (int u = 0; u < kSvSmallSplits; ++u) sum += red[u][c][rr];
        if (ii < T) a_out[(size_t)ii * D + c] = sum * a_scale;
    }
}

template <typename XT>
static cudaError_t launch_svgd_small(int d, const XT* x, int x_ld, int T, const float* score, const GmmParams& G,
                                     int use_gmm, float inv_hs, float hs, float a_scale, float* a_out,
                                     unsigned* status, cudaStream_t st) {
    const dim3 grid((T + kSvSmallRows - 1) / kSvSmallRows), block(kSvSmallThreads);
    const size_t smem = sizeof(float) * 2 * (size_t)d * T;
    switch (d) {
#define COV_SV_SMALL(DD)                                                                                          \
    case DD:                                                                                                    \
        return launch_pdl(svgd_small_kernel<DD, XT>, grid, block, smem, st, x, x_ld, T, score, G, use_gmm, inv_hs, \
                          hs, a_scale, a_out, status);
        COV_SV_SMALL(1) COV_SV_SMALL(2) COV_SV_SMALL(3) COV_SV_SMALL(4) COV_SV_SMALL(5) COV_SV_SMALL(6)
#undef COV_SV_SMALL
    }
    return cudaErrorInvalidValue;
}

// The one-launch Stein field when T <= kSvSmallMaxT (x_double: x points to
// FP64 states), else COV_ERR_UNSUPPORTED.
cov_status svgd_field_small(cov_ctx* ctx, const void* x, bool x_double, int x_ld, int T, int d, const float* score,
                            const cov_gmm* gmm, float h, float* a_out, cudaStream_t stream) {
    // (the staged points and the partial sums within the default 48 KB of shared memory)
    if (T > kSvSmallMaxT || !COV_SVGD_SMALL ||
        sizeof(float) * ((size_t)2 * d * T + (size_t)kSvSmallSplits * d * kSvSmallRows) > 48 * 1024)
        return COV_ERR_UNSUPPORTED;
    if (!ctx || !x || !a_out || T < 1 || d < 1 || d > COV_MAX_D || x_ld < d || !(h > 0.f) || !isfinite(h))
        return COV_ERR_INVALID_ARG;
    GmmParams G{};
    const int use_gmm = score ? 0 : 1;
    if (use_gmm) {
        const cov_status s = make_gmm_params(gmm, d, &G);
        if (s != COV_OK) return s;
    }
    const double r2l = sqrt(2.0 * 0.69314718055994531);
    const float inv_hs = (float)(1.0 / (h * r2l)), hs = (float)(h / r2l), a_scale = (float)(r2l / ((double)h * T));
    const cudaError_t e =
        x_double ? launch_svgd_small(d, static_cast<const double*>(x), x_ld, T, score, G, use_gmm, inv_hs, hs, a_scale,
                                     a_out, ctx->status, stream)
                 : launch_svgd_small(d, static_cast<const float*>(x), x_ld, T, score, G, use_gmm, inv_hs, hs, a_scale,
                                     a_out, ctx->status, stream);
    return cuda_failed(ctx, e) ? COV_ERR_CUDA : COV_OK;
}

struct SvBufs {
    float *xt, *st, *part;
    unsigned* counters;
    int Tp;
};

static SvBufs carve_svgd(Carver& cv, int T, int d) {
    SvBufs B{};
    B.Tp = (int)round_up((size_t)T, kRowPad);
    B.xt = cv.take<float>((size_t)d * B.Tp);
    B.st = cv.take<float>((size_t)d * B.Tp);
    B.counters = cv.take<unsigned>((size_t)B.Tp / 64 + 1);
    B.part = cv.take<float>((size_t)d * (kPartRows + B.Tp));
    return B;
}

size_t svgd_ws_bytes(int T, int d) {
    Carver cv(nullptr);
    carve_svgd(cv, T, d);
    return round_up(cv.off, 256);
}

cov_status svgd_field_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int x_ld, int T, int d,
                         const float* score, const cov_gmm* gmm, float h, float* a_out, cudaStream_t stream) {
    if (!ctx || !x || !a_out || T < 1 || d < 1 || d > COV_MAX_D || x_ld < d || !(h > 0.f) || !isfinite(h))
        return COV_ERR_INVALID_ARG;
    // the workspace the call is documented to need, whichever path runs
    if (!ws || svgd_ws_bytes(T, d) > ws_bytes) return COV_ERR_WORKSPACE;
    {
        const cov_status s = svgd_field_small(ctx, x, false, x_ld, T, d, score, gmm, h, a_out, stream);
        if (s != COV_ERR_UNSUPPORTED) return s;
    }
    GmmParams G{};
    const int use_gmm = score ? 0 : 1;
    if (use_gmm) {
        const cov_status s = make_gmm_params(gmm, d, &G);
        if (s != COV_OK) return s;
    }
    Carver cv(ws);
    SvBufs B = carve_svgd(cv, T, d);
    if (!ws || cv.off > ws_bytes) return COV_ERR_WORKSPACE;
    if (cuda_failed(ctx, cudaMemsetAsync(B.counters, 0, sizeof(unsigned) * (B.Tp / 64 + 1), stream)))
        return COV_ERR_CUDA;
    const double r2l = sqrt(2.0 * 0.69314718055994531);
    launch_pdl(svgd_prep_kernel, dim3((B.Tp + 255) / 256), dim3(256), 0, stream, x, x_ld, T, d, B.Tp, score, G, use_gmm,
                                                             (float)(1.0 / (h * r2l)), (float)(h / r2l), B.xt,
                                                             B.st, ctx->status);
    PairArgs a{};
    a.status = ctx->status;
    a.spin_limit = ctx->spin_limit;
    a.part = B.part;
    a.rows = B.xt; a.row_ld = B.Tp; a.n_rows = T;
    a.cols = B.xt; a.cols2 = B.st; a.col_ld = B.Tp;
    a.a_out = a_out;
    a.a_scale = (float)(r2l / ((double)h * T));
    a.pre_ok = 0;
    const int nc[1] = {T}, co[1] = {0};
    const cov_status r = run_pairs(ctx, d, M_SVGD, &a, nc, 1, co, B.counters, stream);
    if (r != COV_OK) return r;
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

}  // namespace cov

// ---------------------------------------------------------------------------
// C-ABI entry points
// ---------------------------------------------------------------------------
extern "C" cov_status cov_field_sinkhorn_annealed(cov_ctx* ctx, const float* x, int T, const float* y,
                                                  const float* b, int M, int d, float eps, int n_iter,
                                                  float eps_start, float eps_decay, int flags, float* f, float* g,
                                                  float* p, float* a_out, cov_stream_t stream) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::clobber_ws_caches(ctx);  // the workspace scratch overwrites cov_solve's caches
    return cov::sinkhorn_field_ws(ctx, ctx->ws, ctx->ws_bytes, x, d, T, y, b, M, d, eps, n_iter, flags, f, g, p,
                                  a_out, (cudaStream_t)stream, nullptr, eps_start, eps_decay);
}

extern "C" cov_status cov_field_sinkhorn(cov_ctx* ctx, const float* x, int T, const float* y, const float* b, int M,
                                         int d, float eps, int n_iter, int flags, float* f, float* g, float* p,
                                         float* a_out, cov_stream_t stream) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::clobber_ws_caches(ctx);  // the workspace scratch overwrites cov_solve's caches
    return cov::sinkhorn_field_ws(ctx, ctx->ws, ctx->ws_bytes, x, d, T, y, b, M, d, eps, n_iter, flags, f, g, p,
                                  a_out, (cudaStream_t)stream);
}

extern "C" cov_status cov_field_svgd(cov_ctx* ctx, const float* x, int T, int d, const float* score,
                                     const cov_gmm* gmm, float h, float* a_out, cov_stream_t stream) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::clobber_ws_caches(ctx);  // the workspace scratch overwrites cov_solve's caches
    return cov::svgd_field_ws(ctx, ctx->ws, ctx->ws_bytes, x, d, T, d, score, gmm, h, a_out, (cudaStream_t)stream);
}

extern "C" cov_status cov_density_score(cov_ctx* ctx, const float* map, int H, int W, const float* x, int T,
                                        float* score, cov_stream_t stream) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    return cov::density_score_launch(ctx, map, H, W, x, 2, T, score, (cudaStream_t)stream);
}

extern "C" cov_status cov_gmm_score(cov_ctx* ctx, const float* x, int T, int d, const cov_gmm* gmm, float* score,
                                    cov_stream_t stream) {
    if (!ctx || !x || !score || T < 1 || d < 1 || d > COV_MAX_D) return COV_ERR_INVALID_ARG;
    cov::GmmParams G{};
    const cov_status s = cov::make_gmm_params(gmm, d, &G);
    if (s != COV_OK) return s;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    launch_pdl(cov::gmm_score_kernel, dim3((T + 255) / 256), dim3(256), 0, (cudaStream_t)stream, x, T, d, G, score, ctx->status);
    if (cov::cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}
