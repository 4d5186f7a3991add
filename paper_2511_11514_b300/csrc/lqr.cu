// lqr.cu -- control synthesis of Sec. II-C on sm_103a, in FP64:
//   * linearisation A_t = I + dt df/ds, B_t = dt df/du (Eq. 8, Euler map);
//   * the LQR flow-matching problem of Eq. 9-10 on the time grid,
//       min sum_{t=1..T} |z_t - abar_t|_Q^2 + sum_{t=0..T-1} |v_t|_R^2,
//       z_{t+1} = A_t z_t + B_t v_t, z_0 = 0,
//     solved by one warp: a backward Riccati recursion over t = T-1..0
//       S = R + B'P'B, G = B'P'A, h = B'p', K = S^-1 G, k = S^-1 h,
//       P = Q_t + A'P'A - G'K,  p = -Q_t abar_t + A'p' - K'h
//     (P_T = Q, p_T = -Q abar_T, Q_0 = 0) and a forward pass
//       v_t = -K_t z_t - k_t, z_{t+1} = A_t z_t + B_t v_t;
//   * optionally, fused into the forward pass, the control update
//     u_t <- u_t + eta v_t and the rollout s_{t+1} = s_t + dt f(s_t, u_t).
//
// The recursion is a chain of T dependent steps, so it runs on one warp with
// the lanes spread over matrix entries (each lane owns one entry of a
// product per phase, four phases per backward step, two per forward step)
// and the per-step matrices streamed into shared memory one chunk ahead.
#include <math.h>

#include <algorithm>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace cov {

struct LqrConst {
    double Q[COV_MAX_N * COV_MAX_N];
    double R[COV_MAX_M * COV_MAX_M];
};

struct RolloutArgs {
    int model;     // < 0: no update/rollout
    double dt;
    double eta;
    double s0[COV_MAX_N];
    double* u;     // [T][MC] in/out
    double* s;     // [T+1][N] out
};

__device__ __forceinline__ void dyn_f(int model, const double* s, const double* u, double* f) {
    switch (model) {
        case COV_SINGLE_INT:
            f[0] = u[0];
            f[1] = u[1];
            break;
        case COV_DOUBLE_INT:
            f[0] = s[2];
            f[1] = s[3];
            f[2] = u[0];
            f[3] = u[1];
            break;
        default: {  // unicycle
            double sn, cs;
            sincos(s[2], &sn, &cs);
            f[0] = u[0] * cs;
            f[1] = u[0] * sn;
            f[2] = u[1];
        }
    }
}

constexpr int kCh = 32;  // steps per streamed chunk

// Inverse of a small SPD matrix (MC <= 3) by the adjugate; returns false if
// a leading principal minor is not positive.
template <int MC>
__device__ __forceinline__ bool spd_inverse(const double* S, double* Si) {
    if constexpr (MC == 1) {
        Si[0] = 1.0 / S[0];
        return S[0] > 0.0;
    } else if constexpr (MC == 2) {
        const double det = S[0] * S[3] - S[1] * S[2];
        const double inv = 1.0 / det;
        Si[0] = S[3] * inv;
        Si[1] = -S[1] * inv;
        Si[2] = -S[2] * inv;
        Si[3] = S[0] * inv;
        return S[0] > 0.0 && det > 0.0;
    } else {
        const double a = S[0], b = S[1], c = S[2], d = S[3], e = S[4], f = S[5], g = S[6], h = S[7], i = S[8];
        const double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
        const double det = a * A + b * B + c * C;
        const double inv = 1.0 / det;
        Si[0] = A * inv;
        Si[1] = -(b * i - c * h) * inv;
        Si[2] = (b * f - c * e) * inv;
        Si[3] = B * inv;
        Si[4] = (a * i - c * g) * inv;
        Si[5] = -(a * f - c * d) * inv;
        Si[6] = C * inv;
        Si[7] = -(a * h - b * g) * inv;
        Si[8] = (a * e - b * d) * inv;
        return a > 0.0 && (a * e - b * d) > 0.0 && det > 0.0;
    }
}

// Asynchronous 8-byte global->shared copies (cp.async), so the next chunk
// of per-step matrices streams in while the current one is processed.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int N, int MC>
struct LqrSmem {
    double A[2][kCh][N * N];
    double B[2][kCh][N * MC];
    double ab[2][kCh][N];      // backward: targets; forward: unused
    double K[2][kCh][MC * N];  // forward: gains
    double k[2][kCh][MC];
    double u[2][kCh][MC];      // forward: controls (rollout)
    double P[N * N], p[N];
    double PA[N * N], PB[N * MC], h[MC], Atp[N], qa[N];
    double S[MC * MC], G[MC * N], AtPA[N * N];
    double Kc[MC * N], kc[MC];
    double z[N], v[MC], s[N];
};

// Copy `cnt` consecutive rows of `e` doubles starting at row t0 into dst.
__device__ __forceinline__ void stream_rows(double* dst, const double* __restrict__ src, int t0, int cnt, int e,
                                            int lane) {
    for (int i = lane; i < cnt * e; i += 32) cp_async8(dst + i, src + (size_t)t0 * e + i);
}

template <int N, int MC>
__global__ void __launch_bounds__(32, 1) lqr_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                    LqrConst C, const double* __restrict__ abar, int T,
                                                    double* __restrict__ Kg, double* __restrict__ kg,
                                                    double* __restrict__ v_out, double* __restrict__ z_out,
                                                    RolloutArgs ro, unsigned* status) {
    __shared__ __align__(16) LqrSmem<N, MC> sm;
    const int lane = threadIdx.x;
    bool spd_ok = true;

    // P_T = Q, p_T = -Q abar_T
    for (int e = lane; e < N * N; e += 32) sm.P[e] = C.Q[e];
    if (lane < N) {
        double acc = 0.0;
        for (int c = 0; c < N; ++c) acc += C.Q[lane * N + c] * abar[(size_t)(T - 1) * N + c];
        sm.p[lane] = -acc;
    }
    // ---- backward pass: chunk c covers t = lo(c) .. T-1-c*kCh ------------------
    const int n_chunks = (T + kCh - 1) / kCh;
    auto chunk_lo = [&](int c) { return max(0, T - (c + 1) * kCh); };
    auto chunk_cnt = [&](int c) { return T - c * kCh - chunk_lo(c); };
    // abar row for step t is t-1; step t = 0 has no target (zero row)
    auto issue_bwd = [&](int c, int b) {
        const int lo = chunk_lo(c), cnt = chunk_cnt(c);
        stream_rows(&sm.A[b][0][0], A, lo, cnt, N * N, lane);
        stream_rows(&sm.B[b][0][0], B, lo, cnt, N * MC, lane);
        if (lo == 0) {
            if (lane < N) sm.ab[b][0][lane] = 0.0;
            if (cnt > 1) stream_rows(&sm.ab[b][1][0], abar, 0, cnt - 1, N, lane);
        } else {
            stream_rows(&sm.ab[b][0][0], abar, lo - 1, cnt, N, lane);
        }
        cp_async_commit();
    };
    issue_bwd(0, 0);
    for (int c = 0; c < n_chunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < n_chunks) {
            issue_bwd(c + 1, buf ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncwarp();
        const int lo = chunk_lo(c), cnt = chunk_cnt(c);
        for (int j = cnt - 1; j >= 0; --j) {
            const int t = lo + j;
            const double* At = sm.A[buf][j];
            const double* Bt = sm.B[buf][j];
            const double* at = sm.ab[buf][j];
            // phase 1: PA = P'A, PB = P'B, h = B'p'
            for (int e = lane; e < N * N + N * MC + MC; e += 32) {
                if (e < N * N) {
                    const int r = e / N, cc = e % N;
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(sm.P[r * N + q], At[q * N + cc], acc);
                    sm.PA[e] = acc;
                } else if (e < N * N + N * MC) {
                    const int f = e - N * N, r = f / MC, cc = f % MC;
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(sm.P[r * N + q], Bt[q * MC + cc], acc);
                    sm.PB[f] = acc;
                } else {
                    const int r = e - N * N - N * MC;
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(Bt[q * MC + r], sm.p[q], acc);
                    sm.h[r] = acc;
                }
            }
            __syncwarp();
            // phase 2: S = R + B'PB, G = B'PA, AtPA = A'PA, Atp = A'p', qa = Q_t abar_t
            for (int e = lane; e < MC * MC + MC * N + N * N + 2 * N; e += 32) {
                if (e < MC * MC) {
                    const int r = e / MC, cc = e % MC;
                    double acc = C.R[e];
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(Bt[q * MC + r], sm.PB[q * MC + cc], acc);
                    sm.S[e] = acc;
                } else if (e < MC * MC + MC * N) {
                    const int f = e - MC * MC, r = f / N, cc = f % N;
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(Bt[q * MC + r], sm.PA[q * N + cc], acc);
                    sm.G[f] = acc;
                } else if (e < MC * MC + MC * N + N * N) {
                    const int f = e - MC * MC - MC * N, r = f / N, cc = f % N;
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(At[q * N + r], sm.PA[q * N + cc], acc);
                    sm.AtPA[f] = acc;
                } else if (e < MC * MC + MC * N + N * N + N) {
                    const int r = e - MC * MC - MC * N - N * N;
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < N; ++q) acc = fma(At[q * N + r], sm.p[q], acc);
                    sm.Atp[r] = acc;
                } else {
                    const int r = e - MC * MC - MC * N - N * N - N;
                    double acc = 0.0;
                    if (t >= 1) {
#pragma unroll
                        for (int q = 0; q < N; ++q) acc = fma(C.Q[r * N + q], at[q], acc);
                    }
                    sm.qa[r] = acc;
                }
            }
            __syncwarp();
            // phase 3: K = S^-1 G, k = S^-1 h
            if (lane < MC * N + MC) {
                double Si[MC * MC];
                spd_ok &= spd_inverse<MC>(sm.S, Si);
                if (lane < MC * N) {
                    const int r = lane / N, cc = lane % N;
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < MC; ++q) acc = fma(Si[r * MC + q], sm.G[q * N + cc], acc);
                    sm.Kc[lane] = acc;
                    Kg[(size_t)t * MC * N + lane] = acc;
                } else {
                    const int r = lane - MC * N;
                    double acc = 0.0;
#pragma unroll
                    for (int q = 0; q < MC; ++q) acc = fma(Si[r * MC + q], sm.h[q], acc);
                    sm.kc[r] = acc;
                    kg[(size_t)t * MC + r] = acc;
                }
            }
            __syncwarp();
            // phase 4: P = Q_t + A'PA - G'K, p = -Q_t abar_t + A'p' - K'h
            if (lane < N * N) {
                const int r = lane / N, cc = lane % N;
                double acc = sm.AtPA[lane] + (t >= 1 ? C.Q[lane] : 0.0);
#pragma unroll
                for (int q = 0; q < MC; ++q) acc = fma(-sm.G[q * N + r], sm.Kc[q * N + cc], acc);
                sm.P[lane] = acc;
            } else if (lane < N * N + N) {
                const int r = lane - N * N;
                double acc = sm.Atp[r] - sm.qa[r];
#pragma unroll
                for (int q = 0; q < MC; ++q) acc = fma(-sm.Kc[q * N + r], sm.h[q], acc);
                sm.p[r] = acc;
            }
            __syncwarp();
        }
        __syncwarp();
    }
    if (!spd_ok) raise_status(status, kDevNotSpd);
    __threadfence_block();
    __syncwarp();

    // ---- forward pass (+ optional control update and rollout) ----------------
    const bool do_roll = ro.model >= 0;
    if (lane < N) {
        sm.z[lane] = 0.0;
        if (z_out) z_out[lane] = 0.0;
        if (do_roll) {
            sm.s[lane] = ro.s0[lane];
            ro.s[lane] = ro.s0[lane];
        }
    }
    auto issue_fwd = [&](int c, int b) {
        const int t0 = c * kCh, cnt = min(kCh, T - t0);
        stream_rows(&sm.A[b][0][0], A, t0, cnt, N * N, lane);
        stream_rows(&sm.B[b][0][0], B, t0, cnt, N * MC, lane);
        stream_rows(&sm.K[b][0][0], Kg, t0, cnt, MC * N, lane);
        stream_rows(&sm.k[b][0][0], kg, t0, cnt, MC, lane);
        if (do_roll) stream_rows(&sm.u[b][0][0], ro.u, t0, cnt, MC, lane);
        cp_async_commit();
    };
    issue_fwd(0, 0);
    for (int c = 0; c < n_chunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < n_chunks) {
            issue_fwd(c + 1, buf ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncwarp();
        const int t0 = c * kCh, cnt = min(kCh, T - t0);
        for (int j = 0; j < cnt; ++j) {
            const int t = t0 + j;
            // phase F1: v_t = -K_t z_t - k_t
            if (lane < MC) {
                double acc = -sm.k[buf][j][lane];
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(-sm.K[buf][j][lane * N + q], sm.z[q], acc);
                sm.v[lane] = acc;
                v_out[(size_t)t * MC + lane] = acc;
            }
            __syncwarp();
            // phase F2: z_{t+1} = A z + B v (lanes 0..N-1); rollout with the
            // updated control (lanes 8..8+N-1); control write-back (16..16+MC-1)
            double out = 0.0;
            if (lane < N) {
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < N; ++q) acc = fma(sm.A[buf][j][lane * N + q], sm.z[q], acc);
#pragma unroll
                for (int q = 0; q < MC; ++q) acc = fma(sm.B[buf][j][lane * MC + q], sm.v[q], acc);
                out = acc;
            } else if (do_roll && lane >= 8 && lane < 8 + N) {
                double un[MC], f[COV_MAX_N];
#pragma unroll
                for (int q = 0; q < MC; ++q) un[q] = fma(ro.eta, sm.v[q], sm.u[buf][j][q]);
                dyn_f(ro.model, sm.s, un, f);
                out = fma(ro.dt, f[lane - 8], sm.s[lane - 8]);
            } else if (do_roll && lane >= 16 && lane < 16 + MC) {
                ro.u[(size_t)t * MC + (lane - 16)] = fma(ro.eta, sm.v[lane - 16], sm.u[buf][j][lane - 16]);
            }
            __syncwarp();
            if (lane < N) {
                sm.z[lane] = out;
                if (z_out) z_out[(size_t)(t + 1) * N + lane] = out;
            } else if (do_roll && lane >= 8 && lane < 8 + N) {
                sm.s[lane - 8] = out;
                ro.s[(size_t)(t + 1) * N + (lane - 8)] = out;
            }
            __syncwarp();
        }
        __syncwarp();
    }
}

__global__ void linearize_kernel(int model, const double* __restrict__ s, const double* __restrict__ u, int T,
                                 int n, int m, double dt, double* __restrict__ A, double* __restrict__ B) {
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

__global__ void rollout_kernel(int model, RolloutArgs ro, const double* __restrict__ u, int T, int n, int m) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[COV_MAX_N], f[COV_MAX_N];
    for (int r = 0; r < n; ++r) {
        s[r] = ro.s0[r];
        ro.s[r] = s[r];
    }
    for (int t = 0; t < T; ++t) {
        dyn_f(model, s, u + (size_t)t * m, f);
        for (int r = 0; r < n; ++r) {
            s[r] = fma(ro.dt, f[r], s[r]);
            ro.s[(size_t)(t + 1) * n + r] = s[r];
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

size_t lqr_ws_bytes(int T, int n, int m) {
    Carver cv(nullptr);
    cv.take<double>((size_t)T * m * n);
    cv.take<double>((size_t)T * m);
    return round_up(cv.off, 256);
}

template <int N, int MC>
static void launch_lqr_t(const double* A, const double* B, const LqrConst& C, const double* abar, int T, double* Kg,
                         double* kg, double* v, double* z, const RolloutArgs& ro, unsigned* st, cudaStream_t s) {
    lqr_kernel<N, MC><<<1, 32, 0, s>>>(A, B, C, abar, T, Kg, kg, v, z, ro, st);
}

static cov_status launch_lqr(int n, int m, const double* A, const double* B, const LqrConst& C, const double* abar,
                             int T, double* Kg, double* kg, double* v, double* z, const RolloutArgs& ro,
                             unsigned* st, cudaStream_t s) {
#define COV_LQR_CASE(NN, MM)                                               \
    if (n == NN && m == MM) {                                              \
        launch_lqr_t<NN, MM>(A, B, C, abar, T, Kg, kg, v, z, ro, st, s);  \
        return COV_OK;                                                     \
    }
    COV_LQR_CASE(1, 1) COV_LQR_CASE(2, 1) COV_LQR_CASE(3, 1) COV_LQR_CASE(4, 1)
    COV_LQR_CASE(1, 2) COV_LQR_CASE(2, 2) COV_LQR_CASE(3, 2) COV_LQR_CASE(4, 2)
    COV_LQR_CASE(1, 3) COV_LQR_CASE(2, 3) COV_LQR_CASE(3, 3) COV_LQR_CASE(4, 3)
#undef COV_LQR_CASE
    return COV_ERR_UNSUPPORTED;
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

cov_status lqr_track_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const double* A, const double* B, const double* Q,
                        const double* R, const double* abar, int T, int n, int m, double* v_out, double* z_out,
                        cudaStream_t stream) {
    if (!ctx || !A || !B || !abar || !v_out || T < 1 || n < 1 || n > COV_MAX_N || m < 1 || m > COV_MAX_M)
        return COV_ERR_INVALID_ARG;
    LqrConst C;
    if (!make_lqr_const(Q, R, n, m, &C)) return COV_ERR_INVALID_ARG;
    Carver cv(ws);
    double* Kg = cv.take<double>((size_t)T * m * n);
    double* kg = cv.take<double>((size_t)T * m);
    if (!ws || cv.off > ws_bytes) return COV_ERR_WORKSPACE;
    RolloutArgs ro{};
    ro.model = -1;
    const cov_status s = launch_lqr(n, m, A, B, C, abar, T, Kg, kg, v_out, z_out, ro, ctx->status, stream);
    if (s != COV_OK) return s;
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

// Fused LQR + control update + rollout used by cov_solve.
cov_status lqr_update_rollout(cov_ctx* ctx, void* ws, size_t ws_bytes, int model, const double* A, const double* B,
                              const double* Q, const double* R, const double* abar, int T, double dt, double eta,
                              const double* s0, double* u, double* s, double* v, cudaStream_t stream) {
    int n, m;
    if (model_dims(model, &n, &m) != 0) return COV_ERR_INVALID_ARG;
    LqrConst C;
    if (!make_lqr_const(Q, R, n, m, &C)) return COV_ERR_INVALID_ARG;
    Carver cv(ws);
    double* Kg = cv.take<double>((size_t)T * m * n);
    double* kg = cv.take<double>((size_t)T * m);
    if (!ws || cv.off > ws_bytes) return COV_ERR_WORKSPACE;
    RolloutArgs ro{};
    ro.model = model;
    ro.dt = dt;
    ro.eta = eta;
    for (int r = 0; r < n; ++r) ro.s0[r] = s0[r];
    ro.u = u;
    ro.s = s;
    const cov_status st = launch_lqr(n, m, A, B, C, abar, T, Kg, kg, v, nullptr, ro, ctx->status, stream);
    if (st != COV_OK) return st;
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

cov_status linearize_launch(cov_ctx* ctx, int model, const double* s, const double* u, int T, double dt, double* A,
                            double* B, cudaStream_t stream) {
    int n, m;
    if (model_dims(model, &n, &m) != 0) return COV_ERR_INVALID_ARG;
    linearize_kernel<<<(T + 127) / 128, 128, 0, stream>>>(model, s, u, T, n, m, dt, A, B);
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
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::RolloutArgs ro{};
    ro.model = model;
    ro.dt = dt;
    for (int r = 0; r < n; ++r) ro.s0[r] = s0[r];
    ro.s = s;
    cov::rollout_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(model, ro, u, T, n, m);
    if (cov::cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

extern "C" cov_status cov_lqr_track(cov_ctx* ctx, const double* A, const double* B, const double* Q,
                                    const double* R, const double* abar, int T, int n, int m, double* v_out,
                                    double* z_out, cov_stream_t stream) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    return cov::lqr_track_ws(ctx, ctx->ws, ctx->ws_bytes, A, B, Q, R, abar, T, n, m, v_out, z_out,
                             (cudaStream_t)stream);
}
