// lqr.cu -- control synthesis of Sec. II-C on sm_103a, in FP64:
//   * linearisation A_t = I + dt df/ds, B_t = dt df/du (Eq. 8, Euler map);
//   * the LQR flow-matching problem of Eq. 9-10 on the time grid,
//       min sum_{t=1..T} |z_t - abar_t|_Q^2 + sum_{t=0..T-1} |v_t|_R^2,
//       z_{t+1} = A_t z_t + B_t v_t, z_0 = 0,
//     with value function z'P_t z + 2 p_t'z:
//       Riccati (backward, nonlinear in P; per step, one warp):
//         S = R + B'P'B, G = B'P'A, K = S^-1 G, P = Q_t + A'P'A - G'K
//         (P and S kept exactly symmetric: upper triangle computed, mirrored),
//         and the closed loop M_t = A_t - B_t K_t, N_t = S^-1 B_t'
//       affine part (backward, linear in p):
//         p_t = M_t' p_{t+1} + c_t,  c_t = -Q_t abar_t,  p_T = -Q abar_T,
//         k_t = N_t p_{t+1}
//       forward pass (linear in z):
//         z_{t+1} = M_t z_t + e_t,  e_t = -B_t k_t,  v_t = -K_t z_t - k_t
//     (Q_0 = 0; this is the usual recursion written with K'SK = G'K);
//   * the control update u <- u + eta v and the Euler rollout.
//
// FP64 on B300 has a ~65-cycle dependent-FMA latency and ~1.6 FMA/clk per
// SM, so the serial chains are what cost time.  The Riccati recursion runs
// parallel in time by composing its step maps (below; cached for
// time-invariant models), and the two affine recursions as chunked scans:
// each chunk of C steps composes its affine map (one warp per chunk, spread
// over the SMs), one warp chains the chunk maps, and each chunk then fills
// in its steps from its boundary value.  The rollout of every model is a sum of
// Euler increments, done as block-wide prefix sums.  Inside a warp every
// lane runs the same dot product on different operands, so no phase
// diverges.
#include <math.h>

#include <algorithm>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace cov {

struct LqrConst {
    double Q[COV_MAX_N * COV_MAX_N];
    double R[COV_MAX_M * COV_MAX_M];
};

// Cost of one launch in the scan planners' models (us; build flag).
#ifndef COV_SCAN_LAUNCH_US
#define COV_SCAN_LAUNCH_US 1.5
#endif

constexpr int kSB = 32;          // steps per streamed sub-block
constexpr int kMaxChunk = 512;   // steps per scan chunk
constexpr int kMaxChunks = 1024; // scan chunks

// Entry (r, c) of the adjugate of a small symmetric matrix S (MC <= 3):
// (-1)^(r+c) times the minor of S without row c and column r.
template <int MC>
__device__ __forceinline__ double adj_entry(const double* S, int r, int c) {
    if constexpr (MC == 1) {
        return 1.0;
    } else if constexpr (MC == 2) {
        const double v = S[(1 - c) * 2 + (1 - r)];
        return r == c ? v : -v;
    } else {
        const int r0 = c == 0 ? 1 : 0, r1 = c == 2 ? 1 : 2;  // rows of the minor
        const int c0 = r == 0 ? 1 : 0, c1 = r == 2 ? 1 : 2;  // its columns
        const double m = fma(S[r0 * 3 + c0], S[r1 * 3 + c1], -S[r0 * 3 + c1] * S[r1 * 3 + c0]);
        return ((r + c) & 1) ? -m : m;
    }
}
// det(S) of a small SPD matrix; ok &= every leading principal minor > 0.
template <int MC>
__device__ __forceinline__ double spd_det(const double* S, bool& ok) {
    if constexpr (MC == 1) {
        ok &= S[0] > 0.0;
        return S[0];
    } else if constexpr (MC == 2) {
        const double det = fma(S[0], S[3], -S[1] * S[2]);
        ok &= S[0] > 0.0 && det > 0.0;
        return det;
    } else {
        double det = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) det = fma(S[q], adj_entry<3>(S, q, 0), det);
        ok &= S[0] > 0.0 && fma(S[0], S[4], -S[1] * S[3]) > 0.0 && det > 0.0;
        return det;
    }
}

// Copy rows t0 .. t0+cnt-1 (each `e` doubles) of src into dst; thread
// `lane` of `nthreads` takes every nthreads-th double.
__device__ __forceinline__ void stream_rows(double* dst, const double* __restrict__ src, int t0, int cnt, int e,
                                            int lane, int nthreads = 32) {
    for (int i = lane; i < cnt * e; i += nthreads) cp_async8(dst + i, src + (size_t)t0 * e + i);
}

// Sub-blocks of a step range [lo, hi] (inclusive), visited backward or
// forward: sub-block b covers steps first(b) .. first(b)+count(b)-1.
struct SubBlocks {
    int lo, hi, n;
    bool bwd;
    __device__ SubBlocks(int lo_, int hi_, bool b) : lo(lo_), hi(hi_), bwd(b) { n = (hi - lo + kSB) / kSB; }
    __device__ int first(int b) const { return bwd ? max(lo, hi + 1 - (b + 1) * kSB) : lo + b * kSB; }
    __device__ int count(int b) const {
        return bwd ? (hi + 1 - b * kSB) - first(b) : min(kSB, hi + 1 - first(b));
    }
};

// ---------------------------------------------------------------------------
// Riccati recursion (one warp).  Outputs per step: K_t [MC][N], M_t [N][N],
// N_t [MC][N], S_t^-1 [MC][MC] (the last for the adjoint).
// ---------------------------------------------------------------------------
template <int N, int MC>
struct RicSmem {
    double A[2][kSB][N * N];
    double B[2][kSB][N * MC];
    double P[N * N], PA[N * N], PB[N * MC], S[MC * MC], G[MC * N], AtPA[N * N], K[MC * N];
};

// One warp per block.  Pinit == nullptr: block 0 runs t = T-1..0 from
// P_T = Q.  Otherwise block c runs its chunk t = min(T, (c+1) Cc) - 1 .. c Cc
// from the given P entering it, Pinit[c] (the parallel-in-time fill).
template <int N, int MC>
__global__ void __launch_bounds__(32, 1) riccati_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                        LqrConst C, int T, double* __restrict__ Kg,
                                                        double* __restrict__ Mg, double* __restrict__ Ng,
                                                        double* __restrict__ Sg, unsigned* status,
                                                        const double* __restrict__ Pinit, int Cc) {
    pdl_prologue();
    __shared__ __align__(16) RicSmem<N, MC> sm;
    const int lane = threadIdx.x;
    bool spd_ok = true;
    const int lo = Pinit ? blockIdx.x * Cc : 0;
    const int hi = Pinit ? min(T, lo + Cc) - 1 : T - 1;
    for (int e = lane; e < N * N; e += 32) sm.P[e] = Pinit ? Pinit[(size_t)blockIdx.x * N * N + e] : C.Q[e];

    // phase-1 role of this lane: PA = P'A (N*N entries) or PB = P'B (N*MC)
    const bool p1v = lane < N * N + N * MC;
    const bool p1A = lane < N * N;
    const int p1f = p1A ? lane : lane - N * N;
    const int p1w = p1A ? N : MC;
    const int p1r = p1v ? p1f / p1w : 0, p1c = p1v ? p1f % p1w : 0;
    double* p1dst = p1A ? &sm.PA[p1f] : &sm.PB[p1v ? p1f : 0];
    constexpr int NP2 = MC * MC + MC * N + N * N;

    const SubBlocks sb(lo, hi, true);
    auto issue = [&](int b, int buf) {
        stream_rows(&sm.A[buf][0][0], A, sb.first(b), sb.count(b), N * N, lane);
        stream_rows(&sm.B[buf][0][0], B, sb.first(b), sb.count(b), N * MC, lane);
        cp_async_commit();
    };
    issue(0, 0);
    for (int b = 0; b < sb.n; ++b) {
        const int buf = b & 1;
        if (b + 1 < sb.n) {
            issue(b + 1, buf ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncwarp();
        const int t0 = sb.first(b);
        for (int j = sb.count(b) - 1; j >= 0; --j) {
            const int t = t0 + j;
            const double* At = sm.A[buf][j];
            const double* Bt = sm.B[buf][j];
            // phase 1: PA = P'A, PB = P'B
            if (p1v) {
                const double* X = p1A ? At : Bt;
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(sm.P[p1r * N + q], X[q * p1w + p1c], acc);
                *p1dst = acc;
            }
            __syncwarp();
            // phase 2: S = R + B'PB, G = B'PA, AtPA = A'PA
            for (int e = lane; e < NP2; e += 32) {
                const int role = e < MC * MC ? 0 : (e < MC * MC + MC * N ? 1 : 2);
                const int f = e - (role == 0 ? 0 : (role == 1 ? MC * MC : MC * MC + MC * N));
                const int w = role == 0 ? MC : N;
                const int r = f / w, c = f % w;
                const double* Y = role == 2 ? At : Bt;
                const int ys = role == 2 ? N : MC;
                const double* Z = role == 0 ? sm.PB : sm.PA;
                const int zs = role == 0 ? MC : N;
                double acc = role == 0 ? C.R[f] : 0.0;
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(Y[q * ys + r], Z[q * zs + c], acc);
                // S is written from its upper triangle only and mirrored, so it
                // stays exactly symmetric
                double* dst = role == 0 ? &sm.S[f] : (role == 1 ? &sm.G[f] : &sm.AtPA[f]);
                if (role != 0 || r <= c) *dst = acc;
                if (role == 0 && r < c) sm.S[c * MC + r] = acc;
            }
            __syncwarp();
            // phase 3: K = S^-1 G, N_t = S^-1 B', S^-1 -- from the adjugate
            // (adj S) S = det(S) I: each lane forms only the adjugate row its
            // entry needs, its dot product, and one product with 1/det at the
            // end (FP64 instructions are what a step costs on this GPU)
            {
                const double det = spd_det<MC>(sm.S, spd_ok);
                const double inv = 1.0 / det;
                // lanes: K (MC N), N_t (MC N), then S^-1's upper triangle
                // (MC (MC + 1) / 2, mirrored; 30 lanes at most)
                constexpr int NS = MC * (MC + 1) / 2;
                const bool isS = lane >= 2 * MC * N && lane < 2 * MC * N + NS;
                if (lane < 2 * MC * N + NS) {
                    const bool isK = lane < MC * N;
                    const int f = isK ? lane : (isS ? lane - 2 * MC * N : lane - MC * N);
                    // upper-triangle index f -> (r, c), r <= c
                    const int r = isS ? (f < MC ? 0 : (f < 2 * MC - 1 ? 1 : 2)) : f / N;
                    const int c = isS ? f - (r == 0 ? 0 : (r == 1 ? MC - 1 : 2 * MC - 3)) : f % N;
                    double acc = 0.0;
                    if (isS) {
                        acc = adj_entry<MC>(sm.S, r, c);
                    } else {
                        const double* W = isK ? sm.G : Bt;
                        const int ws = isK ? N : 1, wo = isK ? c : c * MC;
#pragma unroll
                        for (int q = 0; q < MC; ++q) acc = fma(adj_entry<MC>(sm.S, r, q), W[q * ws + wo], acc);
                    }
                    const double val = acc * inv;
                    if (isS) {
                        Sg[(size_t)t * MC * MC + r * MC + c] = val;
                        Sg[(size_t)t * MC * MC + c * MC + r] = val;
                    } else {
                        double* g = isK ? Kg : Ng;
                        g[(size_t)t * MC * N + f] = val;
                        if (isK) sm.K[f] = val;
                    }
                }
            }
            __syncwarp();
            // phase 4: P = Q_t + A'PA - G'K, M_t = A - B K
            {
                const bool has_q = t >= 1;
                const bool isP = lane < N * N;
                const int f = isP ? lane : lane - N * N;
                if (lane < 2 * N * N) {
                    const int r = f / N, c = f % N;
                    double acc = isP ? (has_q ? C.Q[f] : 0.0) + sm.AtPA[f] : At[f];
                    const double* U = isP ? sm.G : Bt;
                    const int us = isP ? N : 1, uo = isP ? r : r * MC;
#pragma unroll
                    for (int q = 0; q < MC; ++q) acc = fma(-U[q * us + uo], sm.K[q * N + c], acc);
                    // P from its upper triangle, mirrored: rounding never gives it an
                    // antisymmetric part, which this recursion would amplify
                    if (isP) {
                        if (r <= c) {
                            sm.P[r * N + c] = acc;
                            sm.P[c * N + r] = acc;
                        }
                    } else {
                        Mg[(size_t)t * N * N + f] = acc;
                    }
                }
            }
            __syncwarp();
        }
        __syncwarp();
    }
    if (!spd_ok) raise_status(status, kDevNotSpd);
}

// ---------------------------------------------------------------------------
// Parallel-in-time Riccati.  One step is the map
//   P_t = F_t(P_{t+1}) = Q_t + A_t' P' (I + G_t P')^-1 A_t,  G_t = B_t R^-1 B_t'
// (the Riccati update by the push-through identity).  Maps of the form
// F(P) = J + E' P (I + C P)^-1 E (E square, C and J symmetric PSD) are
// closed under composition: F1(F2(P)) has
//   W = (I + C1 J2)^-1,  E = E2 W E1,  C = C2 + E2 W C1 E2',  J = J1 + (W E1)' J2 E1,
// with every inverse of the form I + (PSD)(PSD), whose eigenvalues are >= 1.
// Chunks compose their maps (one warp each), the chunk maps are chained
// from P_T = Q to get the P entering every chunk (for long horizons through
// grouping levels: groups of maps composed again, level by level, the top
// maps chained, then each group's maps chained from the P entering the
// group, level by level down),
// and each chunk then runs the ordinary Riccati step over its own steps from
// that P (riccati_kernel).
// ---------------------------------------------------------------------------

// B300's FP64 pipe takes one warp-wide FP64 instruction per ~64 clocks per
// warp however many lanes are active (two warps of an SM run in parallel,
// four nearly so), so the serial steps below are written for few FP64
// instructions per warp: each product entry is one lane's dot product, the
// lanes of a warp all work, and where a phase has more than 32 entries a
// second warp takes the rest.
template <int N>
struct RicThreads {
    static constexpr int value = N == 4 ? 64 : 32;
};
template <int NT>
__device__ __forceinline__ void ric_sync() {
    if constexpr (NT == 32)
        __syncwarp();
    else
        __syncthreads();
}

// |x| as an integer key: IEEE magnitudes order like their bit patterns.
__device__ __forceinline__ unsigned long long mag_key(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Solve X Z = Y (X: N x N, N <= 4; Y: N x K) by Gauss-Jordan elimination
// with partial pivoting in division-free form, with the NT threads of the
// block.  aug (N x (N + K), row-major, shared) holds [X | Y] on entry.  At
// pivot k (row p, the largest |aug[r][k]| over r >= k, the first on ties;
// every thread finds it with integer compares) rows k and p trade places
// and every other row r becomes row_r * piv - row_r[k] * row_p: the
// textbook elimination row times piv, the same factor for every row, so the
// pivot choices match the textbook's.  X's part ends diagonal, and
// Z[r][c] = aug[r][N + c] / aug[r][r]: one division per row, all rows at
// once, instead of a reciprocal per pivot on the critical path.  A pivot
// step is two dependent FP64 instructions per thread.  Rows grow by at
// most the pivots' product (for N = 4 bounded by 2^15 M^16 when the entries
// are at most M); a result out of range ends nonfinite and is reported.
template <int N, int K, int NT>
__device__ void block_solve(double* aug, double* Z, int tid) {
    static_assert(N <= 4, "small systems only");
    constexpr int W = N + K, E = N * W, PER = (E + NT - 1) / NT;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int p = k;
        unsigned long long best = mag_key(aug[k * W + k]);
#pragma unroll
        for (int r = k + 1; r < N; ++r) {
            const unsigned long long v = mag_key(aug[r * W + k]);
            if (v > best) {
                best = v;
                p = r;
            }
        }
        const double piv = aug[p * W + k];
        double nv[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + NT * q;
            nv[q] = 0.0;
            if (e < E) {
                const int r = e / W, c = e % W;
                const int src = r == p ? k : r;
                const double pc = aug[p * W + c];
                const double o = fma(aug[src * W + c], piv, -(aug[src * W + k] * pc));
                nv[q] = r == k ? pc : o;
            }
        }
        ric_sync<NT>();
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if (tid + NT * q < E) aug[tid + NT * q] = nv[q];
        ric_sync<NT>();
    }
    for (int e = tid; e < N * K; e += NT) {
        const int r = e / K;
        Z[e] = aug[r * W + N + e % K] / aug[r * W + r];
    }
    ric_sync<NT>();
}

// a0 + sum over q < N of X[q xs] Y[q ys].
template <int N>
__device__ __forceinline__ double dotn(const double* X, int xs, const double* Y, int ys, double a0) {
    double a = a0;
#pragma unroll
    for (int q = 0; q < N; ++q) a = fma(X[q * xs], Y[q * ys], a);
    return a;
}

template <int N>
struct RicMap {
    double E[N * N], C[N * N], J[N * N];
};

template <int N>
struct ComposeScratch {
    double aug[N * 3 * N];  // [X | E1 | C1 E2'] for the solve
    double U[N * N];        // J2 E1
    double VY[N * 2 * N];   // X^-1 [E1 | C1 E2']
};

// acc <- F1 o acc, where F1 = (E1, C1, J1) is the map of the earlier steps
// and acc = (E2, C2, J2) that of the later ones.  With X = I + C1 J2 and
// [V | Y] = X^-1 [E1 | C1 E2'] (one solve):
//   E = E2 V,  C = C2 + E2 Y,  J = J1 + V' (J2 E1)
// (the composition rule above with Y = W C1 E2'), so a step is one product
// level, the solve, and one more product level.  Each product entry is one
// thread's dot product with thread-selected operands (no divergent
// branches).  C and J are symmetric in exact arithmetic and are kept so
// (upper triangle, mirrored).  All NT threads of the block call it.
template <int N, int NT>
__device__ void compose_into(RicMap<N>& acc, const double* E1, const double* C1, const double* J1,
                             ComposeScratch<N>& sc, int tid) {
    constexpr int NN = N * N, W = 3 * N, P = (3 * NN + NT - 1) / NT;
    // X = I + C1 J2 -> aug[:, 0:N], C1 E2' -> aug[:, 2N:3N], U = J2 E1; E1 -> aug[:, N:2N]
    for (int e = tid; e < NN; e += NT) sc.aug[(e / N) * W + N + e % N] = E1[e];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int e = tid + NT * q;
        if (e < 3 * NN) {
            const int which = e / NN, f = e % NN, r = f / N, c = f % N;
            const double* x = which == 2 ? acc.J + r * N : C1 + r * N;
            const double* y = which == 0 ? acc.J + c : (which == 1 ? acc.E + c * N : E1 + c);
            const int ys = which == 1 ? 1 : N;
            double* dst = which == 2 ? sc.U + f : sc.aug + r * W + (which == 0 ? c : 2 * N + c);
            *dst = dotn<N>(x, 1, y, ys, which == 0 && r == c ? 1.0 : 0.0);
        }
    }
    ric_sync<NT>();
    block_solve<N, 2 * N, NT>(sc.aug, sc.VY, tid);
    // E = E2 V, C = C2 + E2 Y, J = J1 + V' U
    double nv[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int e = tid + NT * q;
        nv[q] = 0.0;
        if (e < 3 * NN) {
            const int which = e / NN, f = e % NN, r = f / N, c = f % N;
            const double* x = which == 2 ? sc.VY + r : acc.E + r * N;
            const int xs = which == 2 ? 2 * N : 1;
            const double* y = which == 2 ? sc.U + c : sc.VY + (which == 1 ? N : 0) + c;
            const int ys = which == 2 ? N : 2 * N;
            nv[q] = dotn<N>(x, xs, y, ys, which == 0 ? 0.0 : (which == 1 ? acc.C[f] : J1[f]));
        }
    }
    ric_sync<NT>();
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int e = tid + NT * q;
        if (e < 3 * NN) {
            const int which = e / NN, f = e % NN, r = f / N, c = f % N;
            if (which == 0) {
                acc.E[f] = nv[q];
            } else if (r <= c) {
                double* m = which == 1 ? acc.C : acc.J;
                m[r * N + c] = nv[q];
                m[c * N + r] = nv[q];
            }
        }
    }
    ric_sync<NT>();
}

template <int N, int MC>
struct ComposeSmem {
    double A[2][kSB][N * N];
    double B[2][kSB][N * MC];
    double G[kSB][N * N];  // B_t R^-1 B_t' of the sub-block's steps
    double Qs[N * N], Z0[N * N];
    RicMap<N> acc;
    ComposeScratch<N> sc;
};

// Level 1: block c composes the step maps of chunk c (steps [c Cc,
// min((c+1) Cc, T) - 1]).  The step map is E1 = A_t, C1 = B_t R^-1 B_t',
// J1 = Q_t; the C1 of a whole streamed sub-block are formed together
// before the serial loop, which then only composes.  Launched with
// RicThreads<N>::value threads.
template <int N, int MC>
__global__ void __launch_bounds__(RicThreads<N>::value, 1)
    ric_compose_kernel(const double* __restrict__ A, const double* __restrict__ B, LqrConst Cq, int T, int Cc,
                       double* __restrict__ maps, unsigned* status) {
    pdl_prologue();
    constexpr int NT = RicThreads<N>::value, NN = N * N;
    __shared__ __align__(16) ComposeSmem<N, MC> sm;
    const int tid = threadIdx.x;
    const int lo = blockIdx.x * Cc, hi = min(T, lo + Cc) - 1;
    for (int e = tid; e < NN; e += NT) {
        sm.Qs[e] = Cq.Q[e];
        sm.Z0[e] = 0.0;
    }
    const SubBlocks sb(lo, hi, true);
    auto issue = [&](int b, int buf) {
        stream_rows(&sm.A[buf][0][0], A, sb.first(b), sb.count(b), NN, tid, NT);
        stream_rows(&sm.B[buf][0][0], B, sb.first(b), sb.count(b), N * MC, tid, NT);
        cp_async_commit();
    };
    issue(0, 0);
    bool first = true;
    for (int b = 0; b < sb.n; ++b) {
        const int buf = b & 1;
        if (b + 1 < sb.n) {
            issue(b + 1, buf ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        ric_sync<NT>();
        const int t0 = sb.first(b), cnt = sb.count(b);
        // G_t = B_t R^-1 B_t' (Cq.R holds R^-1), upper triangle mirrored
        for (int e = tid; e < cnt * NN; e += NT) {
            const int j = e / NN, f = e % NN, r = f / N, c = f % N;
            if (r > c) continue;
            const double* Bt = sm.B[buf][j];
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < MC; ++q) {
                double bq = 0.0;
#pragma unroll
                for (int s = 0; s < MC; ++s) bq = fma(Cq.R[q * MC + s], Bt[c * MC + s], bq);
                acc = fma(Bt[r * MC + q], bq, acc);
            }
            sm.G[j][r * N + c] = acc;
            sm.G[j][c * N + r] = acc;
        }
        ric_sync<NT>();
        for (int j = cnt - 1; j >= 0; --j) {
            const int t = t0 + j;
            const double* J1 = t >= 1 ? sm.Qs : sm.Z0;
            if (first) {
                for (int e = tid; e < NN; e += NT) {
                    sm.acc.E[e] = sm.A[buf][j][e];
                    sm.acc.C[e] = sm.G[j][e];
                    sm.acc.J[e] = J1[e];
                }
                first = false;
                ric_sync<NT>();
                continue;
            }
            compose_into<N, NT>(sm.acc, sm.A[buf][j], sm.G[j], J1, sm.sc, tid);
        }
        ric_sync<NT>();
    }
    bool ok = true;
    for (int e = tid; e < NN; e += NT) {
        double* m = maps + (size_t)blockIdx.x * 3 * NN;
        m[e] = sm.acc.E[e];
        m[NN + e] = sm.acc.C[e];
        m[2 * NN + e] = sm.acc.J[e];
        ok &= isfinite(sm.acc.E[e]) && isfinite(sm.acc.C[e]) && isfinite(sm.acc.J[e]);
    }
    if (__syncthreads_or(!ok) && tid == 0) raise_status(status, kDevNonfinite);
}

// Level 2 (long horizons): block g composes the chunk maps [g G, min((g+1)
// G, n_maps) - 1] into one group map, the next map streaming into shared
// memory while the current one is composed.  Launched with
// RicThreads<N>::value threads.
template <int N>
__global__ void __launch_bounds__(RicThreads<N>::value, 1)
    ric_group_kernel(const double* __restrict__ maps, int n_maps, int G, double* __restrict__ out,
                     unsigned* status) {
    pdl_prologue();
    constexpr int NT = RicThreads<N>::value, NN = N * N;
    __shared__ __align__(16) RicMap<N> acc;
    __shared__ __align__(16) double Mb[2][3 * NN];
    __shared__ __align__(16) ComposeScratch<N> sc;
    const int tid = threadIdx.x;
    const int lo = blockIdx.x * G, hi = min(n_maps, lo + G) - 1;
    auto fetch = [&](int k, int buf) {
        for (int e = tid; e < 3 * NN; e += NT) cp_async8(&Mb[buf][e], maps + (size_t)k * 3 * NN + e);
        cp_async_commit();
    };
    fetch(hi, 0);
    for (int k = hi, it = 0; k >= lo; --k, ++it) {
        const int buf = it & 1;
        if (k > lo) {
            fetch(k - 1, buf ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        ric_sync<NT>();
        const double* m = Mb[buf];
        if (k == hi) {
            for (int e = tid; e < NN; e += NT) {
                acc.E[e] = m[e];
                acc.C[e] = m[NN + e];
                acc.J[e] = m[2 * NN + e];
            }
            ric_sync<NT>();
        } else {
            compose_into<N, NT>(acc, m, m + NN, m + 2 * NN, sc, tid);
        }
    }
    bool ok = true;
    for (int e = tid; e < NN; e += NT) {
        double* o = out + (size_t)blockIdx.x * 3 * NN;
        o[e] = acc.E[e];
        o[NN + e] = acc.C[e];
        o[2 * NN + e] = acc.J[e];
        ok &= isfinite(acc.E[e]) && isfinite(acc.C[e]) && isfinite(acc.J[e]);
    }
    if (__syncthreads_or(!ok) && tid == 0) raise_status(status, kDevNonfinite);
}

// Chain maps backward: block b takes the maps [b seg, min((b+1) seg,
// n_maps) - 1] from the P entering its last one (Pstart[b], or P_T = Q when
// Pstart is null) and writes Pin[k] = the P entering map k.  A map is
// applied as P <- J + E' (I + P C)^-1 (P E) (the same value as
// J + E' P (I + C P)^-1 E by the push-through identity; one product level,
// the solve, one more), the next map streaming into shared memory
// meanwhile.
template <int N>
__global__ void __launch_bounds__(32, 1) ric_chain_kernel(const double* __restrict__ maps, int n_maps, int seg,
                                                          const double* __restrict__ Pstart, LqrConst Cq,
                                                          double* __restrict__ Pin, unsigned* status) {
    pdl_prologue();
    constexpr int NN = N * N;
    __shared__ __align__(16) double Mb[2][3 * NN];
    __shared__ double P[NN], V[NN], aug[N * 2 * N];
    const int lane = threadIdx.x;
    const int lo = blockIdx.x * seg, hi = min(n_maps, lo + seg) - 1;
    const bool lo16 = lane < NN;
    const int f = lane % NN, r = f / N, c = f % N;
    if (lo16) P[lane] = Pstart ? Pstart[(size_t)blockIdx.x * NN + lane] : Cq.Q[lane];
    auto fetch = [&](int k, int buf) {
        for (int e = lane; e < 3 * NN; e += 32) cp_async8(&Mb[buf][e], maps + (size_t)k * 3 * NN + e);
        cp_async_commit();
    };
    fetch(hi, 0);
    bool ok = true;
    for (int k = hi, it = 0; k >= lo; --k, ++it) {
        const int buf = it & 1;
        if (k > lo) {
            fetch(k - 1, buf ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncwarp();
        const double* E = Mb[buf];
        const double* Cm = E + NN;
        const double* J = E + 2 * NN;
        // [I + P C | P E] -> aug (lanes [0, NN) the left block, [NN, 2 NN) the right)
        if (lane < 2 * NN) {
            const bool left = lane < NN;
            aug[r * 2 * N + (left ? c : N + c)] =
                dotn<N>(P + r * N, 1, (left ? Cm : E) + c, N, left && r == c ? 1.0 : 0.0);
        }
        if (lo16) Pin[(size_t)k * NN + lane] = P[lane];
        __syncwarp();
        block_solve<N, N, 32>(aug, V, lane);
        double pn = 0.0;
        if (lo16) {  // J + E' V
            pn = dotn<N>(E + r, N, V + c, N, J[f]);
            ok &= isfinite(pn);
        }
        __syncwarp();
        if (lo16 && r <= c) {
            P[r * N + c] = pn;
            P[c * N + r] = pn;
        }
        __syncwarp();
    }
    if (!__all_sync(0xffffffffu, ok) && lane == 0) raise_status(status, kDevNonfinite);
}

// ---------------------------------------------------------------------------
// Affine recursions as chunked scans.  Backward (BWD): p_t = M_t' p_{t+1} +
// c_t for t = T-1..0.  Forward: z_{t+1} = M_t z_t + e_t for t = 0..T-1.
// Chunk c covers steps [c*C, min((c+1)*C, T) - 1].
// ---------------------------------------------------------------------------

// Compose the chunk's affine map (Phi | phi) and write its forcing terms:
//   BWD: c_t = -Q_t abar_t (abar row t-1, t >= 1; c_0 = 0), or c_t = cin[t]
//        when cin is given;                                 map p_lo = Phi p_{hi+1} + phi
//   FWD: e_t = -B_t k_t;                                    map z_{hi+1} = Phi z_lo + phi
template <int N, int MC, bool BWD>
__global__ void __launch_bounds__(32) compose_kernel(const double* __restrict__ Mg, LqrConst Cq,
                                                     const double* __restrict__ abar, const double* __restrict__ Bg,
                                                     const double* __restrict__ kg, const double* __restrict__ cin,
                                                     int T, int C, double* __restrict__ force,
                                                     double* __restrict__ maps) {
    pdl_prologue();
    extern __shared__ __align__(16) double dyn[];
    __shared__ __align__(16) double Ms[2][kSB][N * N];
    __shared__ double X[N * (N + 1)];
    const int lane = threadIdx.x;
    const int lo = blockIdx.x * C, hi = min(lo + C, T) - 1, cnt = hi - lo + 1;
    double* fs = dyn;  // [cnt][N]
    for (int i = lane; i < cnt * N; i += 32) {
        const int t = lo + i / N, r = i % N;
        double acc = 0.0;
        if constexpr (BWD) {
            if (cin) {
                acc = cin[(size_t)t * N + r];
            } else if (t >= 1) {
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(-Cq.Q[r * N + q], abar[(size_t)(t - 1) * N + q], acc);
            }
        } else {
#pragma unroll
            for (int q = 0; q < MC; ++q) acc = fma(-Bg[((size_t)t * N + r) * MC + q], kg[(size_t)t * MC + q], acc);
        }
        fs[i] = acc;
        force[(size_t)t * N + r] = acc;
    }
    constexpr int NX = N * (N + 1);
    const int xr = lane / (N + 1), xc = lane % (N + 1);
    if (lane < NX) X[lane] = (xc == xr) ? 1.0 : 0.0;
    const SubBlocks sb(lo, hi, BWD);
    auto issue = [&](int b, int buf) {
        stream_rows(&Ms[buf][0][0], Mg, sb.first(b), sb.count(b), N * N, lane);
        cp_async_commit();
    };
    issue(0, 0);
    for (int b = 0; b < sb.n; ++b) {
        const int buf = b & 1;
        if (b + 1 < sb.n) {
            issue(b + 1, buf ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncwarp();
        const int t0 = sb.first(b), cntb = sb.count(b);
        for (int jj = 0; jj < cntb; ++jj) {
            const int j = BWD ? cntb - 1 - jj : jj;
            const double* Mt = Ms[buf][j];
            double acc = 0.0;
            if (lane < NX) {
                acc = (xc == N) ? fs[(t0 + j - lo) * N + xr] : 0.0;
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    const double mq = BWD ? Mt[q * N + xr] : Mt[xr * N + q];
                    acc = fma(mq, X[q * (N + 1) + xc], acc);
                }
            }
            __syncwarp();
            if (lane < NX) X[lane] = acc;
            __syncwarp();
        }
        __syncwarp();
    }
    if (lane < NX) maps[(size_t)blockIdx.x * NX + lane] = X[lane];
}

// Chain chunk maps (one warp per block): block b takes the maps [b seg,
// min((b+1) seg, n_maps) - 1] in the scan's direction and writes bnd[c] =
// the value entering chunk c (BWD: p_{hi+1}; FWD: z_lo).  The first value is
// start[b] when start is given (the value entering the block's group), else
// that of the whole recursion: BWD p_T = -Q abar_T or the given w0, FWD 0.
// The block's maps are staged in dynamic shared memory (seg x N x (N+1)).
template <int N, bool BWD>
__global__ void __launch_bounds__(32, 1) boundaries_kernel(const double* __restrict__ maps, int n_maps, int seg,
                                                           const double* __restrict__ start, LqrConst Cq,
                                                           const double* __restrict__ abar,
                                                           const double* __restrict__ w0, int T,
                                                           double* __restrict__ bnd) {
    pdl_prologue();
    extern __shared__ __align__(16) double mp[];  // [seg][N][N+1]
    __shared__ double w[N];
    const int lane = threadIdx.x;
    constexpr int NX = N * (N + 1);
    const int lo = blockIdx.x * seg, cnt = min(n_maps, lo + seg) - lo;
    for (int i = lane; i < cnt * NX; i += 32) cp_async8(mp + i, maps + (size_t)lo * NX + i);
    cp_async_commit();
    if (lane < N) {
        double acc = 0.0;
        if (start) {
            acc = start[(size_t)blockIdx.x * N + lane];
        } else if constexpr (BWD) {
            if (w0) {
                acc = w0[lane];
            } else {
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(-Cq.Q[lane * N + q], abar[(size_t)(T - 1) * N + q], acc);
            }
        }
        w[lane] = acc;
    }
    cp_async_wait_all();
    __syncwarp();
    for (int k = 0; k < cnt; ++k) {
        const int c = BWD ? cnt - 1 - k : k;
        const double* m = mp + (size_t)c * NX;
        double acc = 0.0;
        if (lane < N) {
            bnd[(size_t)(lo + c) * N + lane] = w[lane];
            acc = dotn<N>(m + lane * (N + 1), 1, w, 1, m[lane * (N + 1) + N]);
        }
        __syncwarp();
        if (lane < N) w[lane] = acc;
        __syncwarp();
    }
}

// Level 2 of a long scan: block g composes the chunk maps [g G, min((g+1)
// G, n_maps) - 1] in the scan's direction into one group map (map c after
// the maps before it: (Phi_c Phi | Phi_c phi + phi_c)), the next map
// streaming into shared memory meanwhile.  One warp.
template <int N, bool BWD>
__global__ void __launch_bounds__(32, 1) affine_group_kernel(const double* __restrict__ maps, int n_maps, int G,
                                                             double* __restrict__ out) {
    pdl_prologue();
    constexpr int NX = N * (N + 1);
    __shared__ __align__(16) double Mb[2][NX];
    __shared__ double X[NX];
    const int lane = threadIdx.x;
    const int lo = blockIdx.x * G, cnt = min(n_maps, lo + G) - lo;
    const int xr = lane / (N + 1), xc = lane % (N + 1);
    auto fetch = [&](int k, int buf) {
        const int c = lo + (BWD ? cnt - 1 - k : k);
        if (lane < NX) cp_async8(&Mb[buf][lane], maps + (size_t)c * NX + lane);
        cp_async_commit();
    };
    fetch(0, 0);
    for (int k = 0; k < cnt; ++k) {
        const int buf = k & 1;
        if (k + 1 < cnt) {
            fetch(k + 1, buf ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncwarp();
        const double* m = Mb[buf];
        double acc = 0.0;
        if (lane < NX)
            acc = k == 0 ? m[lane] : dotn<N>(m + xr * (N + 1), 1, X + xc, N + 1, xc == N ? m[xr * (N + 1) + N] : 0.0);
        __syncwarp();
        if (lane < NX) X[lane] = acc;
        __syncwarp();
    }
    if (lane < NX) out[(size_t)blockIdx.x * NX + lane] = X[lane];
}

// Fill the steps of one chunk from its boundary value.
//   BWD: p_t = M_t' p_{t+1} + c_t and k_t = N_t p_{t+1} (+ kx_t when given)
//        -> k [T][MC]; p_0 -> p0_out when given
//   FWD: z_{t+1} = M_t z_t + e_t and v_t = -K_t z_t - k_t   -> v [T][MC], z [T+1][N]
template <int N, int MC, bool BWD>
__global__ void __launch_bounds__(32) fill_kernel(const double* __restrict__ Mg, const double* __restrict__ Wg,
                                                  const double* __restrict__ force, const double* __restrict__ kin,
                                                  const double* __restrict__ bnd, const double* __restrict__ kx,
                                                  int T, int C, double* __restrict__ out_m,
                                                  double* __restrict__ z_out, double* __restrict__ p0_out) {
    pdl_prologue();
    __shared__ __align__(16) double Ms[2][kSB][N * N];
    __shared__ __align__(16) double Ws[2][kSB][MC * N];  // BWD: N_t, FWD: K_t
    __shared__ __align__(16) double Fs[2][kSB][N];
    __shared__ __align__(16) double Ks[2][kSB][MC];      // FWD: k_t
    __shared__ double w[N], wn[N];
    const int lane = threadIdx.x;
    const int lo = blockIdx.x * C, hi = min(lo + C, T) - 1;
    if (lane < N) {
        w[lane] = bnd[(size_t)blockIdx.x * N + lane];
        wn[lane] = -w[lane];
        if (!BWD && z_out && blockIdx.x == 0) z_out[lane] = w[lane];
    }
    const bool isS = lane < N;                 // state lanes
    const bool isO = lane >= N && lane < N + MC;  // output lanes (k or v)
    const int ro = isO ? lane - N : 0;
    const SubBlocks sb(lo, hi, BWD);
    auto issue = [&](int b, int buf) {
        stream_rows(&Ms[buf][0][0], Mg, sb.first(b), sb.count(b), N * N, lane);
        stream_rows(&Ws[buf][0][0], Wg, sb.first(b), sb.count(b), MC * N, lane);
        stream_rows(&Fs[buf][0][0], force, sb.first(b), sb.count(b), N, lane);
        if (!BWD) stream_rows(&Ks[buf][0][0], kin, sb.first(b), sb.count(b), MC, lane);
        cp_async_commit();
    };
    issue(0, 0);
    __syncwarp();
    for (int b = 0; b < sb.n; ++b) {
        const int buf = b & 1;
        if (b + 1 < sb.n) {
            issue(b + 1, buf ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncwarp();
        const int t0 = sb.first(b), cntb = sb.count(b);
        for (int jj = 0; jj < cntb; ++jj) {
            const int j = BWD ? cntb - 1 - jj : jj;
            const int t = t0 + j;
            const double* Mt = Ms[buf][j];
            const double* Wt = Ws[buf][j];
            double acc = 0.0;
            if (isS || isO) {
                // uniform dot: state lanes use M (transposed when BWD) on w;
                // output lanes use W (N_t or K_t) on w (BWD) or -w (FWD)
                const double* X = isS ? Mt : Wt;
                int xs, xo;
                if (isS) {
                    xs = BWD ? N : 1;
                    xo = BWD ? lane : lane * N;
                } else {
                    xs = 1;
                    xo = ro * N;
                }
                const double* wv = (isO && !BWD) ? wn : w;
                acc = isS ? Fs[buf][j][lane] : (BWD ? (kx ? kx[(size_t)t * MC + ro] : 0.0) : -Ks[buf][j][ro]);
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(X[q * xs + xo], wv[q], acc);
            }
            __syncwarp();
            if (isS) {
                w[lane] = acc;
                wn[lane] = -acc;
                if (!BWD && z_out) z_out[(size_t)(t + 1) * N + lane] = acc;
            } else if (isO) {
                out_m[(size_t)t * MC + ro] = acc;
            }
            __syncwarp();
        }
        __syncwarp();
    }
    if (BWD && p0_out && blockIdx.x == 0 && lane < N) p0_out[lane] = w[lane];
}

// ---------------------------------------------------------------------------
// Short horizons: both affine recursions of the LQR step in one CTA.  The
// chunked scans above spread the FP64 work over the SMs but pay a launch per
// level (ten launches for the two recursions at T = 256), which is most of
// their time on a short horizon.  Here lane g of the CTA owns the steps
// [g C, min((g+1) C, T) - 1], C = ceil(T / kShortLanes), and every phase is
// lane-parallel, so each FP64 instruction does useful work in all 32 lanes
// (the FP64 pipe takes one warp instruction per ~64 clocks per warp, about
// four warps at a time per SM):
//   1. every lane composes its chunk's affine map (Phi | phi);
//   2. the maps are chained: an inclusive scan over the lanes of each warp
//      (shuffles, five composition levels), the warps' totals in order by
//      one thread, then each lane applies the scan of the chunks after it
//      (BWD) or before it (FWD) to the value entering its warp;
//   3. every lane runs its steps from the value entering its chunk.
// BWD: p_t = M_t' p_{t+1} + c_t (c_t = -Q abar_{t-1}, c_0 = 0, p_T = -Q abar_T),
//      k_t = N_t p_{t+1} (kept in shared memory for the forward pass);
// FWD: z_0 = 0, z_{t+1} = M_t z_t + e_t (e_t = -B_t k_t), v_t = -K_t z_t - k_t.
// The matrix parts Phi of all these maps depend on the gains alone, so they
// are formed once per set of gains (lqr_short_pre_kernel, launched with the
// Riccati recursion; for a time-invariant model once per solve) and stored
// beside the gains; each LQR step (lqr_short_kernel) then composes and scans
// only the vector parts phi, an N^2 instead of an N^2 (N + 1) FMA product
// per composition.  A composition own o other (other applied first) is
//   Phi = Phi_own Phi_other,  phi = Phi_own phi_other + phi_own,
// and the cache holds, per lane and recursion, Phi_own before each of the
// five scan levels, the Phi of the exclusive scan (the chunks after / before
// the lane's, within its warp) and the warps' total Phi.  Each step's
// arithmetic is that of compose_kernel / fill_kernel, in the same order.
// ---------------------------------------------------------------------------
constexpr int kShortWarps = 4;
constexpr int kShortLanes = 32 * kShortWarps;
constexpr int kShortMaxT = 1024;
constexpr int kShortLevels = 5;                      // log2(32) scan levels
constexpr int kShortLaneMats = kShortLevels + 1;     // + the exclusive scan's Phi
constexpr int kShortRecMats = kShortLanes * kShortLaneMats + kShortWarps;  // per recursion

// Cache matrices (N x N, row-major): recursion r (0 BWD, 1 FWD), lane g,
// slot k (0..4 scan levels, 5 exclusive scan); warp totals after the lanes.
template <int N, class D>
__device__ __forceinline__ D* short_lane_mat(D* cache, int r, int g, int k) {
    return cache + ((size_t)r * kShortRecMats + (size_t)g * kShortLaneMats + k) * N * N;
}
template <int N, class D>
__device__ __forceinline__ D* short_warp_mat(D* cache, int r, int w) {
    return cache + ((size_t)r * kShortRecMats + (size_t)kShortLanes * kShortLaneMats + w) * N * N;
}

template <int N>
__device__ __forceinline__ void mat_identity(double (&P)[N * N]) {
#pragma unroll
    for (int e = 0; e < N * N; ++e) P[e] = (e % (N + 1) == 0) ? 1.0 : 0.0;
}
// P <- P Q
template <int N>
__device__ __forceinline__ void mat_mul_right(double (&P)[N * N], const double (&Q)[N * N]) {
    double R[N * N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < N; ++q) acc = fma(P[i * N + q], Q[q * N + c], acc);
            R[i * N + c] = acc;
        }
#pragma unroll
    for (int e = 0; e < N * N; ++e) P[e] = R[e];
}
template <int N>
__device__ __forceinline__ void mat_shfl(const double (&P)[N * N], double (&Q)[N * N], int off, bool down) {
#pragma unroll
    for (int e = 0; e < N * N; ++e)
        Q[e] = down ? __shfl_down_sync(0xffffffffu, P[e], off) : __shfl_up_sync(0xffffffffu, P[e], off);
}
template <int N>
__device__ __forceinline__ void vec_shfl(const double (&x)[N], double (&y)[N], int off, bool down) {
#pragma unroll
    for (int e = 0; e < N; ++e)
        y[e] = down ? __shfl_down_sync(0xffffffffu, x[e], off) : __shfl_up_sync(0xffffffffu, x[e], off);
}
template <int N>
__device__ __forceinline__ void mat_store(double* dst, const double (&P)[N * N]) {
#pragma unroll
    for (int e = 0; e < N * N; ++e) dst[e] = P[e];
}
// y = P x + b (P from memory)
template <int N>
__device__ __forceinline__ void mat_apply(const double* P, const double* x, const double* b, double* y) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double acc = b[i];
#pragma unroll
        for (int q = 0; q < N; ++q) acc = fma(P[i * N + q], x[q], acc);
        y[i] = acc;
    }
}

// The matrix parts of the short kernel's maps (one CTA of kShortLanes
// threads): BWD chunk map Phi = M_lo' ... M_hi', FWD Phi = M_hi ... M_lo,
// and their warp scans, into `cache`.  M is staged in shared memory first
// (T N^2 <= kShortPreMs).
constexpr int kShortPreMs = 4096;
template <int N>
__global__ void __launch_bounds__(kShortLanes, 1) lqr_short_pre_kernel(const double* __restrict__ Mg, int T,
                                                                       double* __restrict__ cache) {
    pdl_prologue();
    __shared__ double Ms[kShortPreMs];
    const int g = threadIdx.x, lane = g & 31, warp = g >> 5;
    for (int i = g; i < T * N * N; i += kShortLanes) cp_async8(Ms + i, Mg + i);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    const int C = (T + kShortLanes - 1) / kShortLanes;
    const int lo = g * C, hi = min(lo + C, T) - 1;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const bool bwd = r == 0;
        double P[N * N], O[N * N];
        mat_identity<N>(P);
        for (int j = 0; j <= hi - lo; ++j) {  // BWD: t = hi .. lo, P <- M_t' P; FWD: t = lo .. hi, P <- M_t P
            const int t = bwd ? hi - j : lo + j;
            const double* Mt = Ms + t * N * N;
            double R[N * N];
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(bwd ? Mt[q * N + i] : Mt[i * N + q], P[q * N + c], acc);
                    R[i * N + c] = acc;
                }
#pragma unroll
            for (int e = 0; e < N * N; ++e) P[e] = R[e];
        }
#pragma unroll
        for (int k = 0; k < kShortLevels; ++k) {
            const int off = 1 << k;
            mat_store<N>(short_lane_mat<N>(cache, r, g, k), P);
            mat_shfl<N>(P, O, off, bwd);
            if (bwd ? lane + off < 32 : lane >= off) mat_mul_right<N>(P, O);
        }
        mat_shfl<N>(P, O, 1, bwd);
        if (lane == (bwd ? 31 : 0)) mat_identity<N>(O);
        mat_store<N>(short_lane_mat<N>(cache, r, g, kShortLevels), O);
        if (lane == (bwd ? 0 : 31)) mat_store<N>(short_warp_mat<N>(cache, r, warp), P);
    }
}

// Doubles of dynamic shared memory the step kernel stages its inputs in.
__host__ __device__ constexpr size_t short_smem_doubles(int T, int N, int MC) {
    return (size_t)T * (N * N + N + 3 * MC * N + MC) + (size_t)2 * kShortRecMats * N * N;
}

// The single integrator's outer-iteration tail fused into the step kernel
// (ROLL): the field a is lifted while staged, and after the forward pass
// u_t += eta v_t and the Euler rollout s_{t+1} = s_t + dt u_t from s_0 (a
// prefix sum over the lanes, as in update_rollout_kernel).
struct ShortRoll {
    const float* a;  // [T][d] field on the coverage coordinates
    int d;
    double eta, dt;
    double s0[2];
    double* u;       // [T][2] in/out
    double* s;       // [T+1][2] out
};

// One LQR step's affine recursions on the cached matrix parts (one CTA of
// kShortLanes threads; T <= kShortMaxT).  Gains layout as in
// launch_affine_t: M [T][N][N], Nt and K [T][MC][N]; B [T][N][MC].  Every
// input is first staged in shared memory by asynchronous copies in four
// groups, in the order the phases need them (M, abar and the cache; N_t;
// B_t; K_t), so no phase waits on a dependent global load.
template <int N, int MC, bool ROLL>
__global__ void __launch_bounds__(kShortLanes, 1) lqr_short_kernel(const double* __restrict__ Mg,
                                                                   const double* __restrict__ Ng,
                                                                   const double* __restrict__ Kg,
                                                                   const double* __restrict__ Bg, LqrConst Cq,
                                                                   const double* __restrict__ abar, int T,
                                                                   const double* __restrict__ cache,
                                                                   double* __restrict__ v, double* __restrict__ z,
                                                                   ShortRoll ro) {
    static_assert(!ROLL || (N == 2 && MC == 2), "the fused rollout is the single integrator's");
    pdl_prologue();
    extern __shared__ __align__(16) double sm[];
    double* Ms = sm;                                      // [T][N][N]
    double* As = Ms + (size_t)T * N * N;                  // [T][N] abar
    double* Cs = As + (size_t)T * N;                      // the cache
    double* Ns = Cs + (size_t)2 * kShortRecMats * N * N;  // [T][MC][N]
    double* Bs = Ns + (size_t)T * MC * N;                 // [T][N][MC]
    double* Kq = Bs + (size_t)T * N * MC;                 // [T][MC][N]
    double* ks = Kq + (size_t)T * MC * N;                 // [T][MC]: k_t
    __shared__ double tphi[kShortWarps][N];
    __shared__ double xw[kShortWarps][N];
    const int g = threadIdx.x, lane = g & 31, warp = g >> 5;
    auto stage = [&](double* dst, const double* src, int cnt) {
        for (int i = g; i < cnt; i += kShortLanes) cp_async8(dst + i, src + i);
    };
    stage(Ms, Mg, T * N * N);
    if constexpr (ROLL) {
        for (int i = g; i < T * N; i += kShortLanes) {
            const int t = i / N, r = i % N;
            As[i] = r < ro.d ? (double)ro.a[(size_t)t * ro.d + r] : 0.0;
        }
    } else {
        stage(As, abar, T * N);
    }
    stage(Cs, cache, 2 * kShortRecMats * N * N);
    cp_async_commit();
    stage(Ns, Ng, T * MC * N);
    cp_async_commit();
    stage(Bs, Bg, T * N * MC);
    cp_async_commit();
    stage(Kq, Kg, T * MC * N);
    cp_async_commit();
    const int C = (T + kShortLanes - 1) / kShortLanes;
    const int lo = g * C, hi = min(lo + C, T) - 1;  // empty when lo > hi
    // c_t = -Q abar_{t-1} (t >= 1), c_0 = 0
    auto cvec = [&](int t, double* c) {
#pragma unroll
        for (int r = 0; r < N; ++r) {
            double acc = 0.0;
            if (t >= 1) {
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(-Cq.Q[r * N + q], As[(t - 1) * N + q], acc);
            }
            c[r] = acc;
        }
    };
    // e_t = -B_t k_t
    auto evec = [&](int t, double* e) {
#pragma unroll
        for (int r = 0; r < N; ++r) {
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < MC; ++q) acc = fma(-Bs[(t * N + r) * MC + q], ks[t * MC + q], acc);
            e[r] = acc;
        }
    };
    // vector part of the warp scan, the warps' chain (one thread, between
    // two CTA barriers) and the value entering this lane's chunk
    auto chain = [&](int r, double (&phi)[N], double (&in)[N]) {
        const bool bwd = r == 0;
#pragma unroll
        for (int k = 0; k < kShortLevels; ++k) {
            const int off = 1 << k;
            double o[N], y[N];
            vec_shfl<N>(phi, o, off, bwd);
            if (bwd ? lane + off < 32 : lane >= off) {
                mat_apply<N>(short_lane_mat<N>(Cs, r, g, k), o, phi, y);
#pragma unroll
                for (int e = 0; e < N; ++e) phi[e] = y[e];
            }
        }
        double ex[N];
        vec_shfl<N>(phi, ex, 1, bwd);
        if (lane == (bwd ? 31 : 0)) {
#pragma unroll
            for (int e = 0; e < N; ++e) ex[e] = 0.0;
        }
        if (lane == (bwd ? 0 : 31)) {
#pragma unroll
            for (int e = 0; e < N; ++e) tphi[warp][e] = phi[e];
        }
        __syncthreads();
        if (g == 0) {
            double x[N], y[N];
            if (bwd) {
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(-Cq.Q[i * N + q], As[(T - 1) * N + q], acc);
                    x[i] = acc;  // p_T
                }
            } else {
#pragma unroll
                for (int i = 0; i < N; ++i) x[i] = 0.0;  // z_0
            }
#pragma unroll
            for (int j = 0; j < kShortWarps; ++j) {
                const int w = bwd ? kShortWarps - 1 - j : j;
#pragma unroll
                for (int i = 0; i < N; ++i) xw[w][i] = x[i];
                if (j + 1 < kShortWarps) {
                    mat_apply<N>(short_warp_mat<N>(Cs, r, w), x, tphi[w], y);
#pragma unroll
                    for (int i = 0; i < N; ++i) x[i] = y[i];
                }
            }
        }
        __syncthreads();
        mat_apply<N>(short_lane_mat<N>(Cs, r, g, kShortLevels), xw[warp], ex, in);
    };

    // ---- backward recursion ------------------------------------------------
    cp_async_wait_group<3>();
    __syncthreads();
    {
        double phi[N], p[N], np[N];
#pragma unroll
        for (int e = 0; e < N; ++e) phi[e] = 0.0;
        for (int t = hi; t >= lo; --t) {  // phi <- M_t' phi + c_t
            const double* Mt = Ms + t * N * N;
            double c[N];
            cvec(t, c);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                double acc = c[i];
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(Mt[q * N + i], phi[q], acc);
                np[i] = acc;
            }
#pragma unroll
            for (int e = 0; e < N; ++e) phi[e] = np[e];
        }
        chain(0, phi, p);  // p = p_{hi+1}
        cp_async_wait_group<2>();
        __syncthreads();
        for (int t = hi; t >= lo; --t) {
            const double* Mt = Ms + t * N * N;
            const double* Nt = Ns + t * MC * N;
#pragma unroll
            for (int r = 0; r < MC; ++r) {
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(Nt[r * N + q], p[q], acc);
                ks[t * MC + r] = acc;
            }
            double c[N];
            cvec(t, c);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                double acc = c[r];
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(Mt[q * N + r], p[q], acc);
                np[r] = acc;
            }
#pragma unroll
            for (int r = 0; r < N; ++r) p[r] = np[r];
        }
    }
    cp_async_wait_group<1>();
    __syncthreads();

    // ---- forward recursion -------------------------------------------------
    {
        double phi[N], w[N], nw[N];
#pragma unroll
        for (int e = 0; e < N; ++e) phi[e] = 0.0;
        for (int t = lo; t <= hi; ++t) {  // phi <- M_t phi + e_t
            const double* Mt = Ms + t * N * N;
            double e[N];
            evec(t, e);
#pragma unroll
            for (int i = 0; i < N; ++i) {
                double acc = e[i];
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(Mt[i * N + q], phi[q], acc);
                nw[i] = acc;
            }
#pragma unroll
            for (int i = 0; i < N; ++i) phi[i] = nw[i];
        }
        chain(1, phi, w);  // w = z_lo
        cp_async_wait_group<0>();
        __syncthreads();
        if (g == 0 && z) {
#pragma unroll
            for (int r = 0; r < N; ++r) z[r] = 0.0;
        }
        double run[MC];  // ROLL: the chunk's sum of dt u_t (new controls)
#pragma unroll
        for (int r = 0; r < MC; ++r) run[r] = 0.0;
        for (int t = lo; t <= hi; ++t) {
            const double* Mt = Ms + t * N * N;
            const double* Kt = Kq + t * MC * N;
            double vt[MC];
#pragma unroll
            for (int r = 0; r < MC; ++r) {
                double acc = -ks[t * MC + r];
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(Kt[r * N + q], -w[q], acc);
                vt[r] = acc;
                v[(size_t)t * MC + r] = acc;
            }
            double e[N];
            evec(t, e);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                double acc = e[r];
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(Mt[r * N + q], w[q], acc);
                nw[r] = acc;
            }
#pragma unroll
            for (int r = 0; r < N; ++r) {
                w[r] = nw[r];
                if (z) z[(size_t)(t + 1) * N + r] = nw[r];
            }
            if constexpr (ROLL) {
                // u_t += eta v_t; k_t is no longer needed, its slot keeps u_t
#pragma unroll
                for (int r = 0; r < MC; ++r) {
                    const double un = fma(ro.eta, vt[r], ro.u[(size_t)t * MC + r]);
                    ro.u[(size_t)t * MC + r] = un;
                    ks[t * MC + r] = un;
                    run[r] += ro.dt * un;
                }
            }
        }
        if constexpr (ROLL) {
            // exclusive prefix of the chunk sums over the lanes, then each
            // lane's positions s_{t+1} = s_0 + (prefix + running sum)
            double inc[MC];
#pragma unroll
            for (int r = 0; r < MC; ++r) {
                inc[r] = run[r];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double y = __shfl_up_sync(0xffffffffu, inc[r], o);
                    if (lane >= o) inc[r] += y;
                }
                if (lane == 31) tphi[warp][r] = inc[r];
            }
            __syncthreads();
            if (g == 0) {
                double acc[MC];
#pragma unroll
                for (int r = 0; r < MC; ++r) acc[r] = 0.0;
#pragma unroll
                for (int w2 = 0; w2 < kShortWarps; ++w2)
#pragma unroll
                    for (int r = 0; r < MC; ++r) {
                        xw[w2][r] = acc[r];
                        acc[r] += tphi[w2][r];
                    }
#pragma unroll
                for (int r = 0; r < MC; ++r) ro.s[r] = ro.s0[r];
            }
            __syncthreads();
            double acc[MC];
#pragma unroll
            for (int r = 0; r < MC; ++r) acc[r] = xw[warp][r] + (inc[r] - run[r]);
            for (int t = lo; t <= hi; ++t) {
#pragma unroll
                for (int r = 0; r < MC; ++r) {
                    acc[r] += ro.dt * ks[t * MC + r];
                    ro.s[(size_t)(t + 1) * MC + r] = ro.s0[r] + acc[r];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoints.  The LQR solution v(abar) is linear in abar: v = H^-1 G'Q abar
// with z = G v and H = G'QG + R (z_0 = 0), so its VJP abar_bar = Q G H^-1 vbar
// is the same LQR with the linear control cost -2 vbar_t'w_t and no state
// target.  With the gains of the same Riccati recursion:
//   p_T = 0,  p_t = M_t' p_{t+1} + K_t' vbar_t,
//   k_t = N_t p_{t+1} - S_t^-1 vbar_t,
//   z_0 = 0,  z_{t+1} = M_t z_t - B_t k_t,   abar_bar_t = Q z_{t+1}.
// The rollout's VJP is the backward affine recursion
//   lambda_T = sbar_T,  lambda_t = A_t' lambda_{t+1} + sbar_t,  ubar_t = B_t' lambda_{t+1},
// i.e. the same scan with M_t := A_t, N_t := B_t', c_t = sbar_t; s0bar = lambda_0.
// ---------------------------------------------------------------------------
__global__ void lqr_vjp_prep_kernel(const double* __restrict__ K, const double* __restrict__ Si,
                                    const double* __restrict__ vbar, int T, int n, int m, double* __restrict__ c,
                                    double* __restrict__ kx) {
    pdl_prologue();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const double* Kt = K + (size_t)t * m * n;
    const double* St = Si + (size_t)t * m * m;
    const double* vt = vbar + (size_t)t * m;
    for (int r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int q = 0; q < m; ++q) acc = fma(Kt[q * n + r], vt[q], acc);
        c[(size_t)t * n + r] = acc;
    }
    for (int r = 0; r < m; ++r) {
        double acc = 0.0;
        for (int q = 0; q < m; ++q) acc = fma(-St[r * m + q], vt[q], acc);
        kx[(size_t)t * m + r] = acc;
    }
}

__global__ void lqr_vjp_out_kernel(LqrConst C, const double* __restrict__ z, int T, int n, double* __restrict__ out) {
    pdl_prologue();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const double* zt = z + (size_t)(t + 1) * n;
    for (int r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int q = 0; q < n; ++q) acc = fma(C.Q[r * n + q], zt[q], acc);
        out[(size_t)t * n + r] = acc;
    }
}

__global__ void transpose_steps_kernel(const double* __restrict__ B, int T, int n, int m, double* __restrict__ Bt) {
    pdl_prologue();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= T * n * m) return;
    const int t = e / (n * m), f = e % (n * m), r = f / m, q = f % m;  // B_t[r][q] -> Bt_t[q][r]
    Bt[(size_t)t * n * m + q * n + r] = B[e];
}

// ---------------------------------------------------------------------------
// Control update and rollout (one CTA): u_t += eta v_t, then the Euler
// rollout as prefix sums of the increments dt f(s_t, u_t):
//   single integrator: p += dt u
//   double integrator: vel += dt u, then p += dt vel
//   unicycle: theta += dt omega, then x += dt v cos(theta), y += dt v sin(theta)
// ---------------------------------------------------------------------------
struct RolloutArgs {
    int model;
    double dt;
    double eta;
    double s0[COV_MAX_N];
    int heading_only;  // unicycle: stop after the heading (the positions follow in two more kernels)
};

// Block-wide exclusive scan of NV values per thread (1024 threads): on
// return x[c] holds the sum over lower threads and tot[c] the block total.
template <int NV>
__device__ __forceinline__ void block_exclusive_scan(double (&x)[NV], double (&tot)[NV], double (*sh)[NV]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    double inc[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        inc[c] = x[c];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, inc[c], o);
            if (lane >= o) inc[c] += y;
        }
    }
    if (lane == 31)
#pragma unroll
        for (int c = 0; c < NV; ++c) sh[warp][c] = inc[c];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            double w = lane < nw ? sh[lane][c] : 0.0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            sh[lane][c] = w;  // inclusive over warps
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        tot[c] = sh[nw - 1][c];
        x[c] = (inc[c] - x[c]) + (warp > 0 ? sh[warp - 1][c] : 0.0);
    }
    __syncthreads();  // sh is reused by the next scan
}

// u_t += eta v_t and the Euler rollout from s0, in tiles of blockDim x kRK
// steps: each thread owns kRK consecutive steps of a tile (loaded and stored
// as whole rows), the nested prefix sums of the model run in registers
// (thread-serial prefix + block scan of the thread totals) and carry from
// tile to tile.  Increments: single integrator p += dt u; double integrator
// vel += dt u, p += dt vel (vel before its update); unicycle theta += dt
// omega, (x, y) += dt v (cos, sin)(theta before its update).
constexpr int kRK = 4;
constexpr int kUnicycleSplitT = 2048;  // longer unicycle horizons take the three-kernel rollout (without scratch)

__global__ void __launch_bounds__(1024) update_rollout_kernel(RolloutArgs ro, double* __restrict__ u,
                                                               const double* __restrict__ v, int T, int n, int m,
                                                               double* __restrict__ s) {
    pdl_prologue();
    __shared__ double sh[32][2];
    const int tid = threadIdx.x;
    const double dt = ro.dt;
    for (int r = tid; r < n; r += blockDim.x) s[r] = ro.s0[r];
    // carries: state at the start of the tile
    double c0 = ro.s0[0], c1 = ro.s0[1], c2 = n > 2 ? ro.s0[2] : 0.0, c3 = n > 3 ? ro.s0[3] : 0.0;
    const int per_tile = blockDim.x * kRK;
    for (int base = 0; base < T; base += per_tile) {
        const int t0 = base + tid * kRK;
        double uk[kRK][2];
#pragma unroll
        for (int k = 0; k < kRK; ++k) {
            const int t = t0 + k;
            uk[k][0] = uk[k][1] = 0.0;
            if (t < T) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    double w = u[(size_t)t * m + c];
                    if (v) {
                        w = fma(ro.eta, v[(size_t)t * m + c], w);
                        u[(size_t)t * m + c] = w;
                    }
                    uk[k][c] = w;
                }
            }
        }
        double out[kRK][COV_MAX_N];
        if (ro.model == COV_SINGLE_INT || ro.model == COV_DOUBLE_INT) {
            // first level: a_t = dt u_t (positions of the single integrator,
            // velocities of the double integrator)
            double run[2] = {0.0, 0.0}, incl[kRK][2], excl[kRK][2];
#pragma unroll
            for (int k = 0; k < kRK; ++k)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    excl[k][c] = run[c];
                    run[c] += dt * uk[k][c];
                    incl[k][c] = run[c];
                }
            double off[2] = {run[0], run[1]}, tot[2];
            block_exclusive_scan<2>(off, tot, sh);
            const double b0 = ro.model == COV_SINGLE_INT ? c0 : c2, b1 = ro.model == COV_SINGLE_INT ? c1 : c3;
            if (ro.model == COV_SINGLE_INT) {
#pragma unroll
                for (int k = 0; k < kRK; ++k) {
                    out[k][0] = b0 + (off[0] + incl[k][0]);
                    out[k][1] = b1 + (off[1] + incl[k][1]);
                }
                c0 += tot[0];
                c1 += tot[1];
            } else {
                // second level: positions += dt vel_t, vel_t the velocity at time t
                double run2[2] = {0.0, 0.0}, incl2[kRK][2];
#pragma unroll
                for (int k = 0; k < kRK; ++k) {
                    out[k][2] = b0 + (off[0] + incl[k][0]);
                    out[k][3] = b1 + (off[1] + incl[k][1]);
                    run2[0] += dt * (b0 + (off[0] + excl[k][0]));
                    run2[1] += dt * (b1 + (off[1] + excl[k][1]));
                    incl2[k][0] = run2[0];
                    incl2[k][1] = run2[1];
                }
                double off2[2] = {run2[0], run2[1]}, tot2[2];
                block_exclusive_scan<2>(off2, tot2, sh);
#pragma unroll
                for (int k = 0; k < kRK; ++k) {
                    out[k][0] = c0 + (off2[0] + incl2[k][0]);
                    out[k][1] = c1 + (off2[1] + incl2[k][1]);
                }
                c0 += tot2[0];
                c1 += tot2[1];
                c2 += tot[0];
                c3 += tot[1];
            }
        } else {  // unicycle: heading first, then the position increments along it
            double run = 0.0, incl[kRK], excl[kRK];
#pragma unroll
            for (int k = 0; k < kRK; ++k) {
                excl[k] = run;
                run += dt * uk[k][1];
                incl[k] = run;
            }
            double off[1] = {run}, tot[1];
            block_exclusive_scan<1>(off, tot, reinterpret_cast<double(*)[1]>(&sh[0][0]));
            if (ro.heading_only) {
#pragma unroll
                for (int k = 0; k < kRK; ++k) {
                    const int t = t0 + k;
                    if (t < T) s[(size_t)(t + 1) * n + 2] = c2 + (off[0] + incl[k]);
                }
                c2 += tot[0];
                continue;
            }
            double run2[2] = {0.0, 0.0}, incl2[kRK][2];
#pragma unroll
            for (int k = 0; k < kRK; ++k) {
                out[k][2] = c2 + (off[0] + incl[k]);
                double sn, cs;
                sincos(c2 + (off[0] + excl[k]), &sn, &cs);
                const double sp = dt * uk[k][0];
                run2[0] += sp * cs;
                run2[1] += sp * sn;
                incl2[k][0] = run2[0];
                incl2[k][1] = run2[1];
            }
            double off2[2] = {run2[0], run2[1]}, tot2[2];
            block_exclusive_scan<2>(off2, tot2, sh);
#pragma unroll
            for (int k = 0; k < kRK; ++k) {
                out[k][0] = c0 + (off2[0] + incl2[k][0]);
                out[k][1] = c1 + (off2[1] + incl2[k][1]);
            }
            c0 += tot2[0];
            c1 += tot2[1];
            c2 += tot[0];
        }
#pragma unroll
        for (int k = 0; k < kRK; ++k) {
            const int t = t0 + k;
            if (t < T)
#pragma unroll
                for (int r = 0; r < COV_MAX_N; ++r)
                    if (r < n) s[(size_t)(t + 1) * n + r] = out[k][r];
        }
    }
}

// Unicycle rollout for long horizons, second part: the position increments
// dt v_t (cos, sin)(theta_t) of every step in parallel over the whole GPU
// (FP64 sincos is the costly part; one SM would take it serially), written
// into the position slots of row t + 1 for the scan that follows.
__global__ void unicycle_increments_kernel(const double* __restrict__ u, int T, int m, double dt,
                                           double* __restrict__ s) {
    pdl_prologue();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double sn, cs;
    sincos(s[(size_t)t * 3 + 2], &sn, &cs);
    const double sp = dt * u[(size_t)t * m];
    s[(size_t)(t + 1) * 3 + 0] = sp * cs;
    s[(size_t)(t + 1) * 3 + 1] = sp * sn;
}

// Third part: positions as the prefix sums of those increments from the
// initial position (one CTA of tiled block scans, in place).
__global__ void __launch_bounds__(1024) unicycle_positions_kernel(RolloutArgs ro, int T, double* __restrict__ s) {
    pdl_prologue();
    __shared__ double sh[32][2];
    double c0 = ro.s0[0], c1 = ro.s0[1];
    const int per_tile = blockDim.x * kRK;
    for (int base = 0; base < T; base += per_tile) {
        const int t0 = base + threadIdx.x * kRK;
        double inc[kRK][2];
#pragma unroll
        for (int k = 0; k < kRK; ++k) {
            const int t = t0 + k;
            inc[k][0] = t < T ? s[(size_t)(t + 1) * 3 + 0] : 0.0;
            inc[k][1] = t < T ? s[(size_t)(t + 1) * 3 + 1] : 0.0;
        }
        double run[2] = {0.0, 0.0}, incl[kRK][2];
#pragma unroll
        for (int k = 0; k < kRK; ++k) {
            run[0] += inc[k][0];
            run[1] += inc[k][1];
            incl[k][0] = run[0];
            incl[k][1] = run[1];
        }
        double off[2] = {run[0], run[1]}, tot[2];
        block_exclusive_scan<2>(off, tot, sh);
#pragma unroll
        for (int k = 0; k < kRK; ++k) {
            const int t = t0 + k;
            if (t < T) {
                s[(size_t)(t + 1) * 3 + 0] = c0 + (off[0] + incl[k][0]);
                s[(size_t)(t + 1) * 3 + 1] = c1 + (off[1] + incl[k][1]);
            }
        }
        c0 += tot[0];
        c1 += tot[1];
    }
}

// ---------------------------------------------------------------------------
// Long horizons: the rollout's prefix sums chunked over the GPU instead of
// one CTA's FP64 pipe, chunks of kLinChunk steps, one CTA each, two kernels
// per sum.  The sums (`mode`):
//   LIN_SI  single integrator: positions += dt u_t;
//   LIN_DI  double integrator: velocities += dt u_t, positions += dt v_t;
//   UNI_HEAD unicycle heading: theta += dt omega_t;
//   UNI_POS  unicycle positions: += the increments dt v_t (cos, sin)(theta_t)
//            already in s (unicycle_increments_kernel), summed in place.
// The first kernel (applying u += eta v on its chunk where the sum reads u)
// writes the chunk's totals with zero state entering it: A = the sum of its
// increments and, for the double integrator, B = sum dt w_t with w_t the
// velocity gained inside the chunk before step t.  The second recovers the
// state entering its chunk from the earlier chunks' totals (P_c = p_0 +
// sum_{c' < c} A_c', or for the double integrator V_c = v_0 + sum A_c',
// P_c = p_0 + sum (dt len_c' V_c' + B_c'), in one warp) and writes the
// chunk's states.
// ---------------------------------------------------------------------------
constexpr int kLinThreads = 64;
constexpr int kLinChunk = kLinThreads * kRK;  // steps per chunk
constexpr int kLinSplitT = kLinChunk;         // longer horizons take the chunked rollout
enum LinMode { LIN_SI = 0, LIN_DI = 1, UNI_HEAD = 2, UNI_POS = 3 };

// Increment of component c at step t (u already updated).
__device__ __forceinline__ double lin_increment(int mode, const double* __restrict__ u, const double* s, int t, int m,
                                                int n, int c, double dt) {
    if (mode == UNI_POS) return s[(size_t)(t + 1) * n + c];
    if (mode == UNI_HEAD) return c == 0 ? dt * u[(size_t)t * m + 1] : 0.0;
    return dt * u[(size_t)t * m + c];
}

__global__ void __launch_bounds__(kLinThreads) linear_totals_kernel(RolloutArgs ro, int mode, double* __restrict__ u,
                                                                    const double* __restrict__ v, const double* s,
                                                                    int T, int n, int m, double* __restrict__ tot) {
    pdl_prologue();
    __shared__ double sh[32][2];
    const double dt = ro.dt;
    const int t0 = blockIdx.x * kLinChunk + threadIdx.x * kRK;
    double run[2] = {0.0, 0.0}, ex[2] = {0.0, 0.0};
#pragma unroll
    for (int k = 0; k < kRK; ++k) {
        const int t = t0 + k;
        if (t < T) {
            if (v && mode != UNI_POS)
#pragma unroll
                for (int c = 0; c < 2; ++c)
                    u[(size_t)t * m + c] = fma(ro.eta, v[(size_t)t * m + c], u[(size_t)t * m + c]);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                ex[c] += run[c];  // velocity gained before step t (this thread's part)
                run[c] += lin_increment(mode, u, s, t, m, n, c, dt);
            }
        }
    }
    double off[2] = {run[0], run[1]}, totA[2];
    block_exclusive_scan<2>(off, totA, sh);
    const int nv = max(0, min(kRK, T - t0));
    double b[2] = {nv * off[0] + ex[0], nv * off[1] + ex[1]}, totB[2] = {0.0, 0.0};
    if (mode == LIN_DI) block_exclusive_scan<2>(b, totB, sh);
    if (threadIdx.x == 0) {
        double* o = tot + (size_t)blockIdx.x * 4;
        o[0] = totA[0];
        o[1] = totA[1];
        o[2] = dt * totB[0];
        o[3] = dt * totB[1];
    }
}

__global__ void __launch_bounds__(kLinThreads) linear_fill_kernel(RolloutArgs ro, int mode, const double* __restrict__ u,
                                                                  const double* __restrict__ tot, int T, int n, int m,
                                                                  double* s) {
    pdl_prologue();
    __shared__ double sh[32][2];
    __shared__ double carry[4];  // p0 p1 (v0 v1) entering this chunk; the heading in p0
    const bool di = mode == LIN_DI;
    const double dt = ro.dt;
    const int cidx = blockIdx.x, cs = cidx * kLinChunk;
    // the state columns this sum writes: positions (0, 1), or the heading (2)
    const int col0 = mode == UNI_HEAD ? 2 : 0, ncomp = mode == UNI_HEAD ? 1 : 2;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double P[2] = {ro.s0[col0], ncomp > 1 ? ro.s0[col0 + 1] : 0.0};
        double V[2] = {di ? ro.s0[2] : 0.0, di ? ro.s0[3] : 0.0};
        for (int base = 0; base < cidx; base += 32) {
            const int cc = base + lane;
            const bool live = cc < cidx;
            const double len = live ? (double)min(kLinChunk, T - cc * kLinChunk) : 0.0;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const double A = live ? tot[(size_t)cc * 4 + c] : 0.0;
                const double Bt = live ? tot[(size_t)cc * 4 + 2 + c] : 0.0;
                double incl = A;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                // A moves the written columns, except for the double
                // integrator, whose A moves the velocity and whose position
                // moves by dt len V + B over the chunk
                double term = di ? dt * len * (V[c] + (incl - A)) + Bt : A;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
                P[c] += term;
                if (di) V[c] += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        if (lane == 0) {
            carry[0] = P[0];
            carry[1] = P[1];
            carry[2] = V[0];
            carry[3] = V[1];
        }
    }
    if (cidx == 0 && mode != UNI_POS)
        for (int r = threadIdx.x; r < n; r += blockDim.x) s[r] = ro.s0[r];
    __syncthreads();
    const int t0 = cs + threadIdx.x * kRK;
    double run[2] = {0.0, 0.0}, incl[kRK][2], excl[kRK][2];
#pragma unroll
    for (int k = 0; k < kRK; ++k) {
        const int t = t0 + k;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            excl[k][c] = run[c];
            run[c] += t < T ? lin_increment(mode, u, s, t, m, n, c, dt) : 0.0;
            incl[k][c] = run[c];
        }
    }
    double off[2] = {run[0], run[1]}, totA[2];
    block_exclusive_scan<2>(off, totA, sh);  // (its barrier also orders the in-place reads before the writes)
    if (!di) {
#pragma unroll
        for (int k = 0; k < kRK; ++k) {
            const int t = t0 + k;
            if (t < T)
                for (int c = 0; c < ncomp; ++c) s[(size_t)(t + 1) * n + col0 + c] = carry[c] + (off[c] + incl[k][c]);
        }
        return;
    }
    // position: p_{t+1} = P_c + dt (i + 1) V_c + sum_{tau <= i} dt w_tau,
    // w_tau the velocity gained inside the chunk before step tau
    double run2[2] = {0.0, 0.0}, incl2[kRK][2];
#pragma unroll
    for (int k = 0; k < kRK; ++k)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            run2[c] += t0 + k < T ? dt * (off[c] + excl[k][c]) : 0.0;
            incl2[k][c] = run2[c];
        }
    double off2[2] = {run2[0], run2[1]}, tot2[2];
    block_exclusive_scan<2>(off2, tot2, sh);
#pragma unroll
    for (int k = 0; k < kRK; ++k) {
        const int t = t0 + k;
        if (t < T) {
            const double steps = (double)(t - cs + 1);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                s[(size_t)(t + 1) * n + c] = carry[c] + (dt * steps * carry[2 + c] + (off2[c] + incl2[k][c]));
                s[(size_t)(t + 1) * n + 2 + c] = carry[2 + c] + (off[c] + incl[k][c]);
            }
        }
    }
}

__global__ void linearize_kernel(int model, const double* __restrict__ s, const double* __restrict__ u, int T,
                                 int n, int m, double dt, double* __restrict__ A, double* __restrict__ B) {
    pdl_prologue();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double* At = A + (size_t)t * n * n;
    double* Bt = B + (size_t)t * n * m;
    for (int e = 0; e < n * n; ++e) At[e] = (e % (n + 1) == 0) ? 1.0 : 0.0;
    for (int e = 0; e < n * m; ++e) Bt[e] = 0.0;
    const double* st = s + (size_t)t * n;
    const double* ut = u + (size_t)t * m;
    switch (model) {
        case COV_SINGLE_INT:
            Bt[0 * m + 0] = dt;
            Bt[1 * m + 1] = dt;
            break;
        case COV_DOUBLE_INT:
            At[0 * n + 2] = dt;
            At[1 * n + 3] = dt;
            Bt[2 * m + 0] = dt;
            Bt[3 * m + 1] = dt;
            break;
        default: {
            double sn, cs;
            sincos(st[2], &sn, &cs);
            At[0 * n + 2] = -dt * ut[0] * sn;
            At[1 * n + 2] = dt * ut[0] * cs;
            Bt[0 * m + 0] = dt * cs;
            Bt[1 * m + 0] = dt * sn;
            Bt[2 * m + 1] = dt;
        }
    }
}

int model_dims(int model, int* n, int* m) {
    switch (model) {
        case COV_SINGLE_INT: *n = 2; *m = 2; return 0;
        case COV_DOUBLE_INT: *n = 4; *m = 2; return 0;
        case COV_UNICYCLE: *n = 3; *m = 2; return 0;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Chunked scan plan for the affine recursions, with the level structure of
// the parallel Riccati: chunks of C steps compose their maps and later fill
// their steps (one warp each); without grouping one warp chains the chunk
// maps; with `depth` grouping levels groups of G[l] maps of level l are
// composed into level l + 1, one warp chains the top level, and level by
// level down one warp per group chains its maps from the value entering the
// group.  Serial depth C + sum_l G[l] + n[depth] + sum_l G[l] + C steps.
constexpr int kScanMaxGroupLevels = 3;  // grouping levels above the chunks

struct ScanPlan {
    int C, n_chunks;                 // chunks of C steps
    int depth;                       // grouping levels: 0 (one warp chains the chunk maps) .. kScanMaxGroupLevels
    int G[kScanMaxGroupLevels];      // maps per group at each level
    int n[kScanMaxGroupLevels + 1];  // maps at each level (n[0] = n_chunks)
};
// Most chunks a plan for T steps may use (chunks of 8 steps and more, or
// up to 64 chunks for short horizons); with G >= 2 the grouping levels
// together hold at most as many maps again (plus one per level).  The
// scratch is sized by it.
static int scan_chunk_cap(int T) {
    return std::max((T + 7) / 8, std::min(T, 64));
}

// Cost (us) of one serial step of each scan level, and of a launch; the
// chunk levels also pay the FP64 pipe time of the warps sharing an SM
// (~N and ~N + 1 FP64 warp-instructions per step at ~9.4 ns each).
constexpr double kScanComposeUs = 0.25, kScanFillUs = 0.38, kScanGroupUs = 0.3, kScanChainUs = 0.2,
                 kScanLaunchUs = COV_SCAN_LAUNCH_US, kScanComposeWarpUs = 0.037, kScanFillWarpUs = 0.047;
constexpr int kScanSms = 148;  // SMs the cost model assumes

static bool scan_plan_search(int T, ScanPlan* p) {
    double best = 1e300;
    const int c_max = std::min(T, kMaxChunk), cap = scan_chunk_cap(T);
    for (int C = 1; C <= c_max; ++C) {
        const int nc = (T + C - 1) / C;
        if (nc > cap || (C > 1 && (T + C - 2) / (C - 1) == nc)) continue;  // too many, or longer chunks for the same count
        const double w = (double)((nc + kScanSms - 1) / kScanSms);
        const double base = C * (std::max(kScanComposeUs, w * kScanComposeWarpUs) +
                                 std::max(kScanFillUs, w * kScanFillWarpUs)) + 3 * kScanLaunchUs;
        for (int depth = 0; depth <= kScanMaxGroupLevels; ++depth) {
            const int g0 = depth ? (int)pow((double)nc, 1.0 / (depth + 1)) : 0;
            for (int g = std::max(2, g0 - 1); g <= (depth ? g0 + 1 : 2); ++g) {
                ScanPlan pl{};
                pl.C = C;
                pl.n_chunks = nc;
                pl.depth = depth;
                double cost = base;
                int n = nc;
                bool fits = true;
                for (int l = 0; l < depth; ++l) {
                    const int G = std::max(2, std::min(g, n));
                    pl.G[l] = G;
                    pl.n[l] = n;
                    fits &= G <= kMaxChunks;
                    n = (n + G - 1) / G;
                    cost += G * (kScanGroupUs + kScanChainUs) + 2 * kScanLaunchUs;
                }
                pl.n[depth] = n;
                cost += n * kScanChainUs;
                // the one-warp chains stage their maps in shared memory
                if (fits && n <= kMaxChunks && cost < best) {
                    best = cost;
                    *p = pl;
                }
            }
        }
    }
    return best < 1e300;
}

static bool scan_plan(int T, ScanPlan* p) {
    static thread_local int memo_T = -1;
    static thread_local ScanPlan memo;
    static thread_local bool memo_ok = false;
    if (T != memo_T) {
        memo_ok = scan_plan_search(T, &memo);
        memo_T = T;
    }
    *p = memo;
    return memo_ok;
}

// Parallel-in-time Riccati plan.  Level 0: chunks of C1 steps compose
// their step maps (nc1 blocks).  Without grouping one warp chains the nc1
// chunk maps.  With `depth` grouping levels, groups of G[l] maps of level l
// are composed again into the maps of level l + 1 (one block per group),
// one warp chains the top level's maps, and then, level by level down, one
// warp per group chains its own maps from the P entering the group.  Last,
// every chunk runs the ordinary Riccati step over its steps.  Serial depth
// C1 + sum_l G[l] + n[depth] + sum_l G[l] + C1 steps.
// Levels of grouping above the chunks (so up to four levels in all).
constexpr int kRicMaxGroupLevels = 3;

struct RicPlan {
    int C1, nc1;                   // chunks of C1 steps
    int depth;                     // grouping levels: 0 (the chunk maps chained directly) .. kRicMaxGroupLevels
    int G[kRicMaxGroupLevels];     // maps per group at each level
    int n[kRicMaxGroupLevels + 1]; // maps at each level (n[0] = nc1)
};
// Most chunks a plan for T steps may use (chunks of 8 steps and more, or
// up to 64 chunks for short horizons); with G >= 2 every grouping level has
// at most half the maps of the level below, so all levels together at most
// twice the chunks.  The scratch is sized by it.
static int ric_chunk_cap(int T) {
    return std::max((T + 7) / 8, std::min(T, 64));
}

// Scratch maps (each 3 n x n for the map and n x n for the P entering it)
// for a horizon of T steps: chunk maps plus the maps of every grouping level.
static size_t ric_scratch_maps(int T) { return (size_t)2 * ric_chunk_cap(T) + kRicMaxGroupLevels; }

// Cost model (ns) of one serial step of each level: its dependent latency,
// and for the levels that run one warp per chunk the FP64 pipe time a warp
// needs per step (B300: ~1.6 DFMA lanes per clock per SM), which bounds a
// level once several warps share an SM.
// (Measured on B300 at 2032 MHz: a composition step ~1.3 us, a group
// composition ~1.2 us, a chain step ~1.15 us, a Riccati step ~1.45 us; an
// SM retires one FP64 warp-instruction per ~19 clocks, ~20 of them per
// composition step and ~26 per Riccati step.)
constexpr double kRicComposeNs = 1300, kRicComposeWarpNs = 190;
constexpr double kRicStepNs = 1450, kRicStepWarpNs = 245;
constexpr double kRicGroupNs = 1200, kRicChainNs = 1150, kRicLaunchNs = COV_SCAN_LAUNCH_US * 1000;

// Serial cost of chaining nc1 chunk maps through `depth` grouping levels of
// (about) equal group size g: each level composes g maps (group) and later
// chains them again (expand), and the top chains what is left.
static double ric_group_cost(int nc1, int depth, int g, RicPlan* pl) {
    double cost = 0.0;
    int n = nc1;
    for (int l = 0; l < depth; ++l) {
        const int G = std::max(2, std::min(g, n));
        pl->G[l] = G;
        pl->n[l] = n;
        n = (n + G - 1) / G;
        cost += G * (kRicGroupNs + kRicChainNs) + 2 * kRicLaunchNs;
    }
    pl->n[depth] = n;
    pl->depth = depth;
    return cost + n * kRicChainNs;
}

static RicPlan ric_plan(int T, int sms) {
    RicPlan best{};
    double best_cost = 1e300;
    const int c_max = std::min(T, 4096), cap = ric_chunk_cap(T);
    for (int C1 = 1; C1 <= c_max; ++C1) {
        const int nc1 = (T + C1 - 1) / C1;
        if (nc1 > cap || (C1 > 1 && (T + C1 - 2) / (C1 - 1) == nc1)) continue;  // too many, or longer chunks for the same count
        const double w1 = (double)((nc1 + sms - 1) / sms);
        const double lvl1 = C1 * (std::max(kRicComposeNs, w1 * kRicComposeWarpNs) +
                                  std::max(kRicStepNs, w1 * kRicStepWarpNs)) + 3 * kRicLaunchNs;
        for (int depth = 0; depth <= kRicMaxGroupLevels; ++depth) {
            // group size near the depth-th root of the chunk count, and its neighbours
            const int g0 = depth ? (int)pow((double)nc1, 1.0 / (depth + 1)) : 0;
            for (int g = std::max(2, g0 - 1); g <= (depth ? g0 + 1 : 2); ++g) {
                RicPlan pl{};
                pl.C1 = C1;
                pl.nc1 = nc1;
                const double cost = lvl1 + ric_group_cost(nc1, depth, g, &pl);
                if (cost < best_cost) {
                    best_cost = cost;
                    best = pl;
                }
            }
        }
    }
    return best;
}

// Gains per step: K [m][n], M [n][n], N [m][n], S^-1 [m][m]; then the
// parallel Riccati's scratch: per level (chunks, then each grouping level)
// its maps [count][3][n][n] and the P entering each [count][n][n].
// Longest horizon the one-CTA short kernels take for a state dimension.
// Their FP64 work runs on one SM: measured against the chunked scans
// (cov_lqr_track, both in CUDA graphs, random time-varying A_t, before the
// matrix parts were cached) one CTA saved 7-13 us at N = 1 for T = 64-1024
// and 3-10 us at N = 2 for T = 64-512, and lost 11 us at N = 2, T = 1024
// and 1-5 us at N = 3 for T = 64-256.
#ifndef COV_LQR_SHORT
#define COV_LQR_SHORT 1
#endif
#ifndef COV_LQR_SHORT_T1
#define COV_LQR_SHORT_T1 1024
#endif
#ifndef COV_LQR_SHORT_T2
#define COV_LQR_SHORT_T2 512
#endif
#ifndef COV_LQR_SHORT_T3
#define COV_LQR_SHORT_T3 0
#endif
static int short_max_T(int n) {
    if (!COV_LQR_SHORT) return 0;
    return std::min(kShortMaxT, n == 1 ? COV_LQR_SHORT_T1 : (n == 2 ? COV_LQR_SHORT_T2 : (n == 3 ? COV_LQR_SHORT_T3 : 0)));
}
// Dynamic shared memory the step kernel may take (the 227 KB opt-in
// maximum less room for its static arrays).
constexpr size_t kShortSmemMax = (size_t)220 * 1024;
// In range, and the staged inputs fit one CTA's shared memory.
static bool short_ok(int T, int n, int m) {
    return T <= short_max_T(n) && (size_t)T * n * n <= (size_t)kShortPreMs &&
           sizeof(double) * short_smem_doubles(T, n, m) <= kShortSmemMax;
}
// The short kernels' cache of matrix parts, stored after the gains.
static size_t short_cache_doubles(int T, int n, int m) {
    return short_ok(T, n, m) ? (size_t)2 * kShortRecMats * n * n : 0;
}
static size_t gain_base_doubles(int T, int n, int m) {
    return (size_t)T * (2 * (size_t)m * n + (size_t)n * n + (size_t)m * m) + ric_scratch_maps(T) * 4 * n * n;
}

size_t lqr_gain_doubles(int T, int n, int m) { return gain_base_doubles(T, n, m) + short_cache_doubles(T, n, m); }

// Affine scan buffers: forcing terms, k, and the scan scratch (chunk maps
// and boundary values, then the maps and boundary values of the grouping
// levels one after another).
struct AffineBufs {
    double *fc, *fe, *k, *maps, *bnd, *mapsg, *bndg;
};

static AffineBufs carve_affine(Carver& cv, int T, int n, int m) {
    AffineBufs b{};
    const size_t nc = (size_t)scan_chunk_cap(T), ng = nc + kScanMaxGroupLevels;
    b.fc = cv.take<double>((size_t)T * n);
    b.fe = cv.take<double>((size_t)T * n);
    b.k = cv.take<double>((size_t)T * m);
    b.maps = cv.take<double>(nc * n * (n + 1));
    b.bnd = cv.take<double>(nc * n);
    b.mapsg = cv.take<double>(ng * n * (n + 1));
    b.bndg = cv.take<double>(ng * n);
    return b;
}

size_t lqr_ws_bytes(int T, int n, int m) {
    Carver cv(nullptr);
    cv.take<double>(lqr_gain_doubles(T, n, m));
    carve_affine(cv, T, n, m);
    return round_up(cv.off, 256);
}

static bool make_lqr_const(const double* Q, const double* R, int n, int m, LqrConst* C) {
    if (!Q || !R) return false;
    *C = LqrConst{};
    for (int e = 0; e < n * n; ++e) {
        if (!isfinite(Q[e])) return false;
        C->Q[e] = Q[e];
    }
    for (int e = 0; e < m * m; ++e) {
        if (!isfinite(R[e])) return false;
        C->R[e] = R[e];
    }
    return true;
}

// Horizons at least this long use the parallel-in-time Riccati.
constexpr int kParRiccatiMinT = 64;

template <int N, int MC>
static void launch_riccati_t(const double* A, const double* B, const LqrConst& C, const LqrConst& Ci, int T,
                             double* gains, int sms, unsigned* st, cudaStream_t s) {
    double* K = gains;
    double* M = gains + (size_t)T * MC * N;
    double* Nt = M + (size_t)T * N * N;
    double* Si = Nt + (size_t)T * MC * N;
    if (T < kParRiccatiMinT) {
        launch_pdl(riccati_kernel<N, MC>, dim3(1), dim3(32), 0, s, A, B, C, T, K, M, Nt, Si, st, nullptr, T);
        return;
    }
    static thread_local int memo_T = -1, memo_sms = -1;
    static thread_local RicPlan pl;
    if (memo_T != T || memo_sms != sms) {
        pl = ric_plan(T, sms);
        memo_T = T;
        memo_sms = sms;
    }
    // maps and entering P of each level: level 0 the chunks, level l the
    // groups of G[l-1] maps of level l - 1
    constexpr size_t NN = (size_t)N * N;
    double* maps[kRicMaxGroupLevels + 1];
    double* pin[kRicMaxGroupLevels + 1];
    double* p = Si + (size_t)T * MC * MC;
    for (int l = 0; l <= pl.depth; ++l) {
        maps[l] = p;
        pin[l] = maps[l] + (size_t)pl.n[l] * 3 * NN;
        p = pin[l] + (size_t)pl.n[l] * NN;
    }
    launch_pdl(ric_compose_kernel<N, MC>, dim3(pl.nc1), dim3(RicThreads<N>::value), 0, s, A, B, Ci, T, pl.C1, maps[0], st);
    for (int l = 0; l < pl.depth; ++l)
        launch_pdl(ric_group_kernel<N>, dim3(pl.n[l + 1]), dim3(RicThreads<N>::value), 0, s, (const double*)maps[l],
                   pl.n[l], pl.G[l], maps[l + 1], st);
    const int top = pl.depth;
    launch_pdl(ric_chain_kernel<N>, dim3(1), dim3(32), 0, s, (const double*)maps[top], pl.n[top], pl.n[top],
               (const double*)nullptr, C, pin[top], st);
    for (int l = top - 1; l >= 0; --l)
        launch_pdl(ric_chain_kernel<N>, dim3(pl.n[l + 1]), dim3(32), 0, s, (const double*)maps[l], pl.n[l], pl.G[l],
                   (const double*)pin[l + 1], C, pin[l], st);
    launch_pdl(riccati_kernel<N, MC>, dim3(pl.nc1), dim3(32), 0, s, A, B, C, T, K, M, Nt, Si, st,
               (const double*)pin[0], pl.C1);
}

// The short kernels' matrix parts from fresh gains (horizons they take).
template <int N, int MC>
static void launch_short_pre_t(double* gains, int T, cudaStream_t s) {
    if constexpr (N <= 3) {
        if (short_ok(T, N, MC)) {
            const double* M = gains + (size_t)T * MC * N;
            launch_pdl(lqr_short_pre_kernel<N>, dim3(1), dim3(kShortLanes), 0, s, M, T,
                       gains + gain_base_doubles(T, N, MC));
        }
    }
}

// R^-1 on the host (m <= 3, Gauss-Jordan with partial pivoting).
static bool invert_small(const double* R, int m, double* Ri) {
    double a[COV_MAX_M][2 * COV_MAX_M];
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < 2 * m; ++c) a[r][c] = c < m ? R[r * m + c] : (c - m == r ? 1.0 : 0.0);
    for (int k = 0; k < m; ++k) {
        int p = k;
        for (int r = k + 1; r < m; ++r)
            if (fabs(a[r][k]) > fabs(a[p][k])) p = r;
        if (!(fabs(a[p][k]) > 0.0)) return false;
        for (int c = 0; c < 2 * m; ++c) std::swap(a[k][c], a[p][c]);
        const double iv = 1.0 / a[k][k];
        for (int c = 0; c < 2 * m; ++c) a[k][c] *= iv;
        for (int r = 0; r < m; ++r) {
            if (r == k) continue;
            const double f = a[r][k];
            for (int c = 0; c < 2 * m; ++c) a[r][c] -= f * a[k][c];
        }
    }
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) Ri[r * m + c] = a[r][m + c];
    return true;
}

// The boundary values of one chunked scan from its chunk maps (ab.maps ->
// ab.bnd), in two or three levels as planned.
template <int N, bool BWD>
static void launch_boundaries(const ScanPlan& pl, const AffineBufs& ab, const LqrConst& C, const double* abar,
                              const double* w0, int T, cudaStream_t s) {
    constexpr size_t NX = (size_t)N * (N + 1);
    // maps and boundary values of each level: level 0 the chunks
    double* maps[kScanMaxGroupLevels + 1] = {ab.maps};
    double* bnd[kScanMaxGroupLevels + 1] = {ab.bnd};
    double* pm = ab.mapsg;
    double* pb = ab.bndg;
    for (int l = 1; l <= pl.depth; ++l) {
        maps[l] = pm;
        bnd[l] = pb;
        pm += (size_t)pl.n[l] * NX;
        pb += (size_t)pl.n[l] * N;
    }
    for (int l = 0; l < pl.depth; ++l)
        launch_pdl(affine_group_kernel<N, BWD>, dim3(pl.n[l + 1]), dim3(32), 0, s, (const double*)maps[l], pl.n[l],
                   pl.G[l], maps[l + 1]);
    const int top = pl.depth;
    launch_pdl(boundaries_kernel<N, BWD>, dim3(1), dim3(32), sizeof(double) * pl.n[top] * NX, s,
               (const double*)maps[top], pl.n[top], pl.n[top], (const double*)nullptr, C, abar, w0, T, bnd[top]);
    for (int l = top - 1; l >= 0; --l)
        launch_pdl(boundaries_kernel<N, BWD>, dim3(pl.n[l + 1]), dim3(32), sizeof(double) * pl.G[l] * NX, s,
                   (const double*)maps[l], pl.n[l], pl.G[l], (const double*)bnd[l + 1], C, abar, w0, T, bnd[l]);
}

template <int N, int MC>
static void launch_affine_t(const double* B, const double* gains, const LqrConst& C, const double* abar, int T,
                            const ScanPlan& pl, const AffineBufs& ab, double* v, double* z, cudaStream_t s) {
    const double* K = gains;
    const double* M = gains + (size_t)T * MC * N;
    const double* Nt = M + (size_t)T * N * N;
    if constexpr (N <= 3) {
        if (short_ok(T, N, MC)) {
            const double* cache = gains + gain_base_doubles(T, N, MC);
            launch_pdl(lqr_short_kernel<N, MC, false>, dim3(1), dim3(kShortLanes),
                       sizeof(double) * short_smem_doubles(T, N, MC), s, M, Nt, K, B, C, abar, T, cache, v, z,
                       ShortRoll{});
            return;
        }
    }
    const size_t fsb = sizeof(double) * pl.C * N;
    launch_pdl(compose_kernel<N, MC, true>, dim3(pl.n_chunks), dim3(32), fsb, s, M, C, abar, nullptr, nullptr, nullptr, T, pl.C, ab.fc,
                                                             ab.maps);
    launch_boundaries<N, true>(pl, ab, C, abar, nullptr, T, s);
    launch_pdl(fill_kernel<N, MC, true>, dim3(pl.n_chunks), dim3(32), 0, s, M, Nt, ab.fc, nullptr, ab.bnd, nullptr, T, pl.C, ab.k, nullptr,
                                                        nullptr);
    launch_pdl(compose_kernel<N, MC, false>, dim3(pl.n_chunks), dim3(32), fsb, s, M, C, nullptr, B, ab.k, nullptr, T, pl.C, ab.fe,
                                                              ab.maps);
    launch_boundaries<N, false>(pl, ab, C, nullptr, nullptr, T, s);
    launch_pdl(fill_kernel<N, MC, false>, dim3(pl.n_chunks), dim3(32), 0, s, M, K, ab.fe, ab.k, ab.bnd, nullptr, T, pl.C, v, z, nullptr);
}

template <int N, int MC>
static void set_attrs_t() {
    const int big = (int)(sizeof(double) * kMaxChunks * N * (N + 1));
    cudaFuncSetAttribute(boundaries_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(boundaries_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if constexpr (N <= 3) {
        if (short_max_T(N) > 0)
            cudaFuncSetAttribute(lqr_short_kernel<N, MC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::min<size_t>(sizeof(double) * short_smem_doubles(short_max_T(N), N, MC),
                                                       kShortSmemMax));
        if constexpr (N == 2 && MC == 2) {
            if (short_max_T(N) > 0)
                cudaFuncSetAttribute(lqr_short_kernel<N, MC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::min<size_t>(sizeof(double) * short_smem_doubles(short_max_T(N), N, MC),
                                                           kShortSmemMax));
        }
    }
}

#define COV_LQR_DISPATCH(MACRO) \
    MACRO(1, 1) MACRO(2, 1) MACRO(3, 1) MACRO(4, 1) MACRO(1, 2) MACRO(2, 2) MACRO(3, 2) MACRO(4, 2) \
    MACRO(1, 3) MACRO(2, 3) MACRO(3, 3) MACRO(4, 3)

void lqr_set_attributes() {
#define COV_ATTR_CASE(NN, MM) set_attrs_t<NN, MM>();
    COV_LQR_DISPATCH(COV_ATTR_CASE)
#undef COV_ATTR_CASE
    cudaGetLastError();
}

cov_status lqr_riccati(cov_ctx* ctx, int n, int m, const double* A, const double* B, const double* Q,
                       const double* R, int T, double* gains, cudaStream_t stream) {
    LqrConst C;
    if (!make_lqr_const(Q, R, n, m, &C)) return COV_ERR_INVALID_ARG;
    LqrConst Ci = C;  // the compose kernel takes R^-1 in place of R
    if (!invert_small(R, m, Ci.R)) return COV_ERR_INVALID_ARG;
#define COV_RIC_CASE(NN, MM)                                                      \
    if (n == NN && m == MM) {                                                     \
        launch_riccati_t<NN, MM>(A, B, C, Ci, T, gains, ctx->num_sms, ctx->status, stream);     \
        launch_short_pre_t<NN, MM>(gains, T, stream);                             \
        return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;     \
    }
    COV_LQR_DISPATCH(COV_RIC_CASE)
#undef COV_RIC_CASE
    return COV_ERR_UNSUPPORTED;
}

cov_status lqr_affine(cov_ctx* ctx, void* ws, size_t ws_bytes, int n, int m, const double* B, const double* gains,
                      const double* Q, const double* abar, int T, double* v_out, double* z_out,
                      cudaStream_t stream) {
    LqrConst C;
    const double R1[COV_MAX_M * COV_MAX_M] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (!make_lqr_const(Q, R1, n, m, &C)) return COV_ERR_INVALID_ARG;
    ScanPlan pl;
    if (!scan_plan(T, &pl)) return COV_ERR_UNSUPPORTED;
    Carver cv(ws);
    const AffineBufs ab = carve_affine(cv, T, n, m);
    if (!ws || cv.off > ws_bytes) return COV_ERR_WORKSPACE;
#define COV_AFF_CASE(NN, MM)                                                          \
    if (n == NN && m == MM) {                                                         \
        launch_affine_t<NN, MM>(B, gains, C, abar, T, pl, ab, v_out, z_out, stream);  \
        return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;         \
    }
    COV_LQR_DISPATCH(COV_AFF_CASE)
#undef COV_AFF_CASE
    return COV_ERR_UNSUPPORTED;
}

// The single integrator's LQR step, control update and rollout in one
// launch (short horizons): a [T][d] the field (lifted inside), v [T][2]
// written, u [T][2] updated, s [T+1][2] the new trajectory from s0.
// COV_ERR_UNSUPPORTED outside the short kernel's range (the caller then
// runs the lift, lqr_affine and update_rollout).
cov_status lqr_step_single_int(cov_ctx* ctx, const double* B, const double* gains, const double* Q, const float* a,
                               int d, int T, double* v, double eta, double dt, const double* s0, double* u, double* s,
                               cudaStream_t stream) {
    constexpr int N = 2, MC = 2;
    if (!short_ok(T, N, MC) || d < 1 || d > N) return COV_ERR_UNSUPPORTED;
    LqrConst C;
    const double R1[COV_MAX_M * COV_MAX_M] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (!make_lqr_const(Q, R1, N, MC, &C)) return COV_ERR_INVALID_ARG;
    const double* K = gains;
    const double* M = gains + (size_t)T * MC * N;
    const double* Nt = M + (size_t)T * N * N;
    const double* cache = gains + gain_base_doubles(T, N, MC);
    ShortRoll ro{};
    ro.a = a;
    ro.d = d;
    ro.eta = eta;
    ro.dt = dt;
    ro.s0[0] = s0[0];
    ro.s0[1] = s0[1];
    ro.u = u;
    ro.s = s;
    launch_pdl(lqr_short_kernel<N, MC, true>, dim3(1), dim3(kShortLanes), sizeof(double) * short_smem_doubles(T, N, MC),
               stream, M, Nt, K, B, C, (const double*)nullptr, T, cache, v, (double*)nullptr, ro);
    return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;
}

cov_status lqr_track_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const double* A, const double* B, const double* Q,
                        const double* R, const double* abar, int T, int n, int m, double* v_out, double* z_out,
                        cudaStream_t stream) {
    if (!ctx || !A || !B || !abar || !v_out || T < 1 || n < 1 || n > COV_MAX_N || m < 1 || m > COV_MAX_M)
        return COV_ERR_INVALID_ARG;
    LqrConst C;
    if (!make_lqr_const(Q, R, n, m, &C)) return COV_ERR_INVALID_ARG;
    ScanPlan pl;
    if (!scan_plan(T, &pl)) return COV_ERR_UNSUPPORTED;
    Carver cv(ws);
    double* gains = cv.take<double>(lqr_gain_doubles(T, n, m));
    const size_t used = round_up(cv.off, 256);
    if (!ws || used > ws_bytes) return COV_ERR_WORKSPACE;
    cov_status s = lqr_riccati(ctx, n, m, A, B, Q, R, T, gains, stream);
    if (s != COV_OK) return s;
    return lqr_affine(ctx, static_cast<char*>(ws) + used, ws_bytes - used, n, m, B, gains, Q, abar, T, v_out, z_out,
                      stream);
}

struct AdjScanBufs {
    AffineBufs ab;
    double *c, *kx, *vtmp, *z, *zero, *Bt;
};

static AdjScanBufs carve_adj_scan(Carver& cv, int T, int n, int m) {
    AdjScanBufs b{};
    b.ab = carve_affine(cv, T, n, m);
    b.c = cv.take<double>((size_t)T * n);
    b.kx = cv.take<double>((size_t)T * m);
    b.vtmp = cv.take<double>((size_t)T * m);
    b.z = cv.take<double>((size_t)(T + 1) * n);
    b.zero = cv.take<double>(COV_MAX_N);
    b.Bt = cv.take<double>((size_t)T * n * m);
    return b;
}

size_t lqr_adj_ws_bytes(int T, int n, int m) {
    Carver cv(nullptr);
    carve_adj_scan(cv, T, n, m);
    return round_up(cv.off, 256);
}

template <int N, int MC>
static void launch_lqr_vjp_t(const double* B, const double* gains, const LqrConst& C, const double* vbar, int T,
                             const ScanPlan& pl, const AdjScanBufs& b, double* out, cudaStream_t s) {
    const double* K = gains;
    const double* M = gains + (size_t)T * MC * N;
    const double* Nt = M + (size_t)T * N * N;
    const double* Si = Nt + (size_t)T * MC * N;
    const size_t fsb = sizeof(double) * pl.C * N;
    const AffineBufs& ab = b.ab;
    launch_pdl(lqr_vjp_prep_kernel, dim3((T + 127) / 128), dim3(128), 0, s, K, Si, vbar, T, N, MC, b.c, b.kx);
    launch_pdl(compose_kernel<N, MC, true>, dim3(pl.n_chunks), dim3(32), fsb, s, M, C, nullptr, nullptr, nullptr, b.c, T, pl.C, ab.fc,
                                                             ab.maps);
    launch_boundaries<N, true>(pl, ab, C, nullptr, b.zero, T, s);
    launch_pdl(fill_kernel<N, MC, true>, dim3(pl.n_chunks), dim3(32), 0, s, M, Nt, ab.fc, nullptr, ab.bnd, b.kx, T, pl.C, ab.k, nullptr,
                                                        nullptr);
    launch_pdl(compose_kernel<N, MC, false>, dim3(pl.n_chunks), dim3(32), fsb, s, M, C, nullptr, B, ab.k, nullptr, T, pl.C, ab.fe,
                                                              ab.maps);
    launch_boundaries<N, false>(pl, ab, C, nullptr, nullptr, T, s);
    launch_pdl(fill_kernel<N, MC, false>, dim3(pl.n_chunks), dim3(32), 0, s, M, K, ab.fe, ab.k, ab.bnd, nullptr, T, pl.C, b.vtmp, b.z,
                                                         nullptr);
    launch_pdl(lqr_vjp_out_kernel, dim3((T + 127) / 128), dim3(128), 0, s, C, b.z, T, N, out);
}

template <int N, int MC>
static void launch_rollout_vjp_t(const double* A, const double* B, const double* sbar, int T, const ScanPlan& pl,
                                 const AdjScanBufs& b, double* ubar, double* s0bar, cudaStream_t s) {
    const size_t fsb = sizeof(double) * pl.C * N;
    const AffineBufs& ab = b.ab;
    const LqrConst C{};
    launch_pdl(transpose_steps_kernel, dim3((T * N * MC + 255) / 256), dim3(256), 0, s, B, T, N, MC, b.Bt);
    launch_pdl(compose_kernel<N, MC, true>, dim3(pl.n_chunks), dim3(32), fsb, s, A, C, nullptr, nullptr, nullptr, sbar, T, pl.C, ab.fc,
                                                             ab.maps);
    launch_boundaries<N, true>(pl, ab, C, nullptr, sbar + (size_t)T * N, T, s);
    launch_pdl(fill_kernel<N, MC, true>, dim3(pl.n_chunks), dim3(32), 0, s, A, b.Bt, ab.fc, nullptr, ab.bnd, nullptr, T, pl.C, ubar,
                                                        nullptr, s0bar);
}

cov_status lqr_vjp_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, int n, int m, const double* B, const double* gains,
                      const double* Q, const double* vbar, int T, double* abar_bar, cudaStream_t stream) {
    LqrConst C;
    const double R1[COV_MAX_M * COV_MAX_M] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (!make_lqr_const(Q, R1, n, m, &C)) return COV_ERR_INVALID_ARG;
    ScanPlan pl;
    if (!scan_plan(T, &pl)) return COV_ERR_UNSUPPORTED;
    Carver cv(ws);
    const AdjScanBufs b = carve_adj_scan(cv, T, n, m);
    if (!ws || cv.off > ws_bytes) return COV_ERR_WORKSPACE;
    if (cuda_failed(ctx, cudaMemsetAsync(b.zero, 0, sizeof(double) * COV_MAX_N, stream))) return COV_ERR_CUDA;
#define COV_LVJP_CASE(NN, MM)                                                            \
    if (n == NN && m == MM) {                                                            \
        launch_lqr_vjp_t<NN, MM>(B, gains, C, vbar, T, pl, b, abar_bar, stream);         \
        return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;            \
    }
    COV_LQR_DISPATCH(COV_LVJP_CASE)
#undef COV_LVJP_CASE
    return COV_ERR_UNSUPPORTED;
}

cov_status rollout_vjp_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, int n, int m, const double* A, const double* B,
                          const double* sbar, int T, double* ubar, double* s0bar, cudaStream_t stream) {
    ScanPlan pl;
    if (!scan_plan(T, &pl)) return COV_ERR_UNSUPPORTED;
    Carver cv(ws);
    const AdjScanBufs b = carve_adj_scan(cv, T, n, m);
    if (!ws || cv.off > ws_bytes) return COV_ERR_WORKSPACE;
#define COV_RVJP_CASE(NN, MM)                                                              \
    if (n == NN && m == MM) {                                                              \
        launch_rollout_vjp_t<NN, MM>(A, B, sbar, T, pl, b, ubar, s0bar, stream);           \
        return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;              \
    }
    COV_LQR_DISPATCH(COV_RVJP_CASE)
#undef COV_RVJP_CASE
    return COV_ERR_UNSUPPORTED;
}

size_t rollout_scratch_doubles(int T) { return (size_t)4 * ((T + kLinChunk - 1) / kLinChunk); }

// scratch (rollout_scratch_doubles(T), may be null): the chunk totals of the
// chunked rollout of the linear models at long horizons (without it they
// roll out in one CTA).
cov_status update_rollout(cov_ctx* ctx, int model, const double* s0, double* u, const double* v, double eta, int T,
                          double dt, double* s, cudaStream_t stream, double* scratch) {
    int n, m;
    if (model_dims(model, &n, &m) != 0) return COV_ERR_INVALID_ARG;
    RolloutArgs ro{};
    ro.model = model;
    ro.dt = dt;
    ro.eta = eta;
    for (int r = 0; r < n; ++r) ro.s0[r] = s0[r];
    if (T > kLinSplitT && scratch) {
        const int nc = (T + kLinChunk - 1) / kLinChunk;
        auto sum = [&](int mode, const double* vv) {
            launch_pdl(linear_totals_kernel, dim3(nc), dim3(kLinThreads), 0, stream, ro, mode, u, vv, (const double*)s,
                       T, n, m, scratch);
            launch_pdl(linear_fill_kernel, dim3(nc), dim3(kLinThreads), 0, stream, ro, mode, (const double*)u,
                       (const double*)scratch, T, n, m, s);
        };
        if (model == COV_UNICYCLE) {
            // heading, then the increments along it, then their sums
            sum(UNI_HEAD, v);
            launch_pdl(unicycle_increments_kernel, dim3((T + 255) / 256), dim3(256), 0, stream, (const double*)u, T, m,
                       dt, s);
            sum(UNI_POS, nullptr);
        } else {
            sum(model == COV_DOUBLE_INT ? LIN_DI : LIN_SI, v);
        }
        return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;
    }
    // as many warps as the horizon fills (kRK steps per thread), up to 1024
    // threads: short horizons scan over fewer warps
    const int threads = std::min(1024, std::max(32, ((T + kRK - 1) / kRK + 31) / 32 * 32));
    // without scratch for the chunked sums, long unicycle horizons still
    // spread the per-step sincos over the GPU: the heading scan, the
    // increments, then the position scan, each scan in one CTA
    ro.heading_only = model == COV_UNICYCLE && T > kUnicycleSplitT;
    launch_pdl(update_rollout_kernel, dim3(1), dim3(threads), 0, stream, ro, u, v, T, n, m, s);
    if (ro.heading_only) {
        launch_pdl(unicycle_increments_kernel, dim3((T + 255) / 256), dim3(256), 0, stream, (const double*)u, T, m,
                   dt, s);
        launch_pdl(unicycle_positions_kernel, dim3(1), dim3(threads), 0, stream, ro, T, s);
    }
    return cuda_failed(ctx, cudaGetLastError()) ? COV_ERR_CUDA : COV_OK;
}

cov_status linearize_launch(cov_ctx* ctx, int model, const double* s, const double* u, int T, double dt, double* A,
                            double* B, cudaStream_t stream) {
    int n, m;
    if (model_dims(model, &n, &m) != 0) return COV_ERR_INVALID_ARG;
    launch_pdl(linearize_kernel, dim3((T + 127) / 128), dim3(128), 0, stream, model, s, u, T, n, m, dt, A, B);
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

}  // namespace cov

extern "C" cov_status cov_linearize(cov_ctx* ctx, int model, const double* s, const double* u, int T, double dt,
                                    double* A, double* B, cov_stream_t stream) {
    int n, m;
    if (!ctx || !s || !u || !A || !B || T < 1 || !isfinite(dt) || cov::model_dims(model, &n, &m) != 0)
        return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    return cov::linearize_launch(ctx, model, s, u, T, dt, A, B, (cudaStream_t)stream);
}

extern "C" cov_status cov_rollout(cov_ctx* ctx, int model, const double* s0, const double* u, int T, double dt,
                                  double* s, cov_stream_t stream) {
    int n, m;
    if (!ctx || !s0 || !u || !s || T < 1 || !isfinite(dt) || cov::model_dims(model, &n, &m) != 0)
        return COV_ERR_INVALID_ARG;
    for (int r = 0; r < n; ++r)
        if (!isfinite(s0[r])) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    // the workspace, when reserved, holds the chunked rollout's totals
    double* scratch = nullptr;
    if (ctx->ws && ctx->ws_bytes >= sizeof(double) * cov::rollout_scratch_doubles(T)) {
        cov::clobber_ws_caches(ctx);
        scratch = static_cast<double*>(ctx->ws);
    }
    return cov::update_rollout(ctx, model, s0, const_cast<double*>(u), nullptr, 0.0, T, dt, s, (cudaStream_t)stream,
                               scratch);
}

extern "C" cov_status cov_lqr_track(cov_ctx* ctx, const double* A, const double* B, const double* Q,
                                    const double* R, const double* abar, int T, int n, int m, double* v_out,
                                    double* z_out, cov_stream_t stream) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::clobber_ws_caches(ctx);  // the workspace scratch overwrites cov_solve's caches
    return cov::lqr_track_ws(ctx, ctx->ws, ctx->ws_bytes, A, B, Q, R, abar, T, n, m, v_out, z_out,
                             (cudaStream_t)stream);
}

extern "C" size_t cov_workspace_size_lqr_vjp(int T, int n, int m) {
    if (T < 1 || n < 1 || n > COV_MAX_N || m < 1 || m > COV_MAX_M) return 0;
    const size_t gains = cov::round_up(sizeof(double) * cov::lqr_gain_doubles(T, n, m), 256);
    const size_t lin = cov::round_up(sizeof(double) * (size_t)T * n * n, 256) +
                       cov::round_up(sizeof(double) * (size_t)T * n * m, 256);
    return std::max(gains, lin) + cov::lqr_adj_ws_bytes(T, n, m) + 4096;
}

extern "C" cov_status cov_lqr_vjp(cov_ctx* ctx, const double* A, const double* B, const double* Q, const double* R,
                                  const double* vbar, int T, int n, int m, double* abar_bar, cov_stream_t stream) {
    if (!ctx || !A || !B || !Q || !R || !vbar || !abar_bar || T < 1 || n < 1 || n > COV_MAX_N || m < 1 ||
        m > COV_MAX_M)
        return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::clobber_ws_caches(ctx);  // the workspace scratch overwrites cov_solve's caches
    cov::Carver cv(ctx->ws);
    double* gains = cv.take<double>(cov::lqr_gain_doubles(T, n, m));
    const size_t used = cov::round_up(cv.off, 256);
    if (!ctx->ws || used > ctx->ws_bytes) return COV_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    cov_status s = cov::lqr_riccati(ctx, n, m, A, B, Q, R, T, gains, st);
    if (s != COV_OK) return s;
    return cov::lqr_vjp_ws(ctx, static_cast<char*>(ctx->ws) + used, ctx->ws_bytes - used, n, m, B, gains, Q, vbar, T,
                           abar_bar, st);
}

extern "C" cov_status cov_rollout_vjp(cov_ctx* ctx, int model, const double* s, const double* u, int T, double dt,
                                      const double* sbar, double* ubar, double* s0bar, cov_stream_t stream) {
    int n, m;
    if (!ctx || !s || !u || !sbar || !ubar || !s0bar || T < 1 || !isfinite(dt) ||
        cov::model_dims(model, &n, &m) != 0)
        return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::clobber_ws_caches(ctx);  // the workspace scratch overwrites cov_solve's caches
    cov::Carver cv(ctx->ws);
    double* A = cv.take<double>((size_t)T * n * n);
    double* B = cv.take<double>((size_t)T * n * m);
    const size_t used = cov::round_up(cv.off, 256);
    if (!ctx->ws || used > ctx->ws_bytes) return COV_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    cov_status r = cov::linearize_launch(ctx, model, s, u, T, dt, A, B, st);
    if (r != COV_OK) return r;
    return cov::rollout_vjp_ws(ctx, static_cast<char*>(ctx->ws) + used, ctx->ws_bytes - used, n, m, A, B, sbar, T,
                               ubar, s0bar, st);
}
