// tc_records.cuh -- column records of the tensor-core exponent kernel
// (lse_tc.cuh): the TF32 parts of each point's prescaled coordinates and of
// its per-column term h, laid out as the K-major core matrices that a
// kind::tf32 MMA reads.  Internal header of libcov.
#pragma once

#include "cov_device.cuh"

namespace cov {

constexpr int kTcRows = 128;                       // rows per CTA (MMA M)
#ifndef COV_TC_COLS
#define COV_TC_COLS 256
#endif
#ifndef COV_TC_READERS
#define COV_TC_READERS 16
#endif
constexpr int kTcCols = COV_TC_COLS;               // columns per tile (MMA N)
constexpr int kTcStages = 2;                       // shared-memory ring of column tiles
constexpr int kTcSoftWarps = COV_TC_READERS;       // accumulator readers: 4 lane quarters x (kTcCols / 64) column groups
static_assert(kTcSoftWarps * 16 == kTcCols, "each reader warp takes 32 lanes x 64 columns of a tile");
constexpr int kTcColGroups = kTcSoftWarps / 4;     // column groups of a tile, 64 columns each
constexpr int kTcThreads = 32 * (kTcSoftWarps + 1);
constexpr int kTcTmemCols = 2 * kTcCols;           // two accumulator buffers (all 512 columns of the SM)
constexpr int kTcMinBlocks = 512 / kTcTmemCols;    // resident CTAs per SM that tensor memory allows
// Launch size from which the automatic setting takes the tensor cores: there
// the tensor-core kernel measured 7-10 % faster than the CUDA-core one, below
// it slower (one 544-thread CTA per SM is too coarse for short launches).
constexpr long long kTcAutoPairs = 1LL << 30;
// Of the 64 exponentials a reader thread takes per tile, how many pairs go
// to the FMA pipe (exp2_fma2) instead of MUFU (build flag
// -DCOV_TC_POLY_PAIRS=0..32).  Default 1: at T = 65536, M = 262144 the
// kernel ran at 0.741 of the MUFU rate with 1 pair (3 %), 0.737 with none
// and 0.733 with 2 -- the readers are not bound by MUFU alone, and the
// polynomial's ~8 instructions per value soon cost more than they free.
#ifndef COV_TC_POLY_PAIRS
#define COV_TC_POLY_PAIRS 1
#endif
constexpr int kTcPolyPairs = COV_TC_POLY_PAIRS;
constexpr int kTcRecC = 8;                         // floats per point in the coordinate record
constexpr int kTcRecH = 4;                         // floats per point in the h record
constexpr unsigned kTcTileBytes = kTcCols * (kTcRecC + kTcRecH) * 4;

// Coordinate record / A-operand layout: point j, slot k (0..7) -> float index.
// Groups of 8 points are 256 bytes: the core matrix of slots 0-3 (8 points x
// 16 bytes), then that of slots 4-7.
__host__ __device__ constexpr int tc_rec_index(int j, int k) {
    return (j >> 3) * 64 + (k >> 2) * 32 + (j & 7) * 4 + (k & 3);
}


// The h record of one point: the three TF32 parts of h and, for d = 3, the
// high part of its third coordinate (its row-side partner is X2l).
template <int D>
__device__ __forceinline__ float4 tc_hrec(float h, float c2) {
    float4 r;
    r.x = tf32r(h);
    r.y = tf32r(h - r.x);
    r.z = tf32r(h - r.x - r.y);
    r.w = D == 3 ? tf32r(c2) : 0.f;
    return r;
}

// Column-side coordinate slots of one point (c = its prescaled coordinates).
template <int D>
__device__ __forceinline__ void tc_crec(const float* c, float (&s)[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = 0.f;
#pragma unroll
    for (int k = 0; k < (D < 2 ? D : 2); ++k) {
        const float hi = tf32r(c[k]), lo = tf32r(c[k] - hi);
        s[3 * k] = hi;
        s[3 * k + 1] = lo;
        s[3 * k + 2] = hi;
    }
    if constexpr (D == 3) {
        const float hi = tf32r(c[2]);
        s[6] = hi;
        s[7] = tf32r(c[2] - hi);
    }
}

}  // namespace cov
