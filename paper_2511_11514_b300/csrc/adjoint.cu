// adjoint.cu -- reverse mode of the Sinkhorn-divergence field (Eq. 5-7)
// through its n_iter unrolled log-domain iterations, on sm_103a.
//
// The forward record (sinkhorn_tape_ws) keeps the per-column terms of every
// iteration, so every softmax of the forward can be rebuilt with a FIXED
// normaliser; e.g. for the f-update of iteration t
//     pi^f_ij = 2^(hy^t_j + 2 xhat_i.yhat_j + hx^t_i - log2 a)   (<= 1),
//     pi^g_ji = 2^(hx^{t-1}_i + 2 xhat_i.yhat_j + hy^t_j - log2 b_j),
//     pi^p_ik = 2^(hp^{t-1}_k + 2 xhat_i.xhat_k - L_i),  L_i = log2 a + hp^{t-1}_i - 2 hp^t_i.
// Every reverse step is therefore an all-pairs weighted sum
//     O_r = sum_c 2^(alpha_r + beta_c + 2 xhat_r.xhat_c) V_c
// without a running maximum (the exponent never exceeds 0 beyond rounding).
// With the adjoints in natural units (fbar = dL/df etc.) the reverse
// iteration t = n..1 is
// (V is staged pre-multiplied, so a pair costs the exponent and 1 + d FMAs)
//   f-step (rows j over columns i, V_i = fbar_i [1, xhat_i]):
//     gbar_j = -W_j,  lbbar_j -= eps W_j,
//     ybar_j += 2 sigma (yhat_j W_j - X_j) - 2 sigma gbar_j Dg^t_j
//   g-step (rows i over columns j, V_j = gbar_j [1, yhat_j]):
//     fbar_i = -W_i,  xbar_i += 2 sigma (xhat_i W_i - Y_i) - 2 sigma fbar_i Df^{t-1}_i
//   p-step (rows k over columns i, V_i = pbar_i/2 [1, xhat_i]):
//     pbar'_k = pbar_k/2 - W_k,  xbar_k += 2 sigma (xhat_k W_k - X_k) - sigma pbar_k Dp^t_k
// where D^t are the barycentric offsets each forward update recorded of its
// own softmax (the row sums of the reverse step), and sigma = sqrt(eps ln 2).
// Before the loop the field itself is differentiated (A_i = 2 abar_i):
//   row pass (rows i): the softmax covariance C_i of yhat (resp. xhat), then
//     xbar_i += 2 ln2 C_i A_i and Gamma_i = A_i . (barycentre of row i);
//   column pass (rows j over columns i) with u_ij = A_i.yhat_j - Gamma_i:
//     ybar_j += sum_i pi_ij A_i - 2 ln2 sum_i pi_ij u_ij (yhat_j - xhat_i),
//     gbar_j = sigma/eps sum_i pi_ij u_ij,  lbbar_j += sigma sum_i pi_ij u_ij,
//   and the same for the self term with -A_i, pi^s and pbar.
// The weights enter through lb_j = log(b_j / sum b):
//   bbar_k = lbbar_k / b_k - (sum_j lbbar_j) / sum b.
#include <math.h>

#include <algorithm>

#include "cov_device.cuh"
#include "cov_internal.h"

namespace cov {

enum AdjKind { A_COL = 0, A_MOM = 1, A_FCOL = 2 };
enum AdjEpi { E_FREV = 0, E_GREV = 1, E_PREV = 2, E_MOM_CROSS = 3, E_MOM_SELF = 4, E_FCOL_CROSS = 5, E_FCOL_SELF = 6 };

constexpr int kATile = 256;   // columns per staged tile
constexpr int kAWarps = 4;    // warps per CTA, each takes a quarter of a tile
constexpr int kAThreads = 32 * kAWarps;
constexpr int kAMaxSlots = 1536;
constexpr size_t kAPartRows = (size_t)2 * kAMaxSlots * 128 + 1024;

// Per kind: rows per lane R, staged floats per column NC, accumulators NACC.
template <int D, int KIND>
struct AdjTraits;
template <int D>
struct AdjTraits<D, A_COL> {
    static constexpr int R = 4, NC = 2 * D + 2, NACC = D + 1;
};
template <int D>
struct AdjTraits<D, A_MOM> {
    static constexpr int R = 2, NC = D + 1, NACC = 1 + D + D * (D + 1) / 2;
};
template <int D>
struct AdjTraits<D, A_FCOL> {
    static constexpr int R = 2, NC = 2 * D + 2, NACC = 1 + 2 * D;
};

struct AdjArgs {
    // rows: coordinates [D][row_ld]; exponent term alpha_i = ca ra[i] + cb rb[i] + c0
    const float* rows;
    int row_ld;
    int n_rows;
    const float* ra;
    const float* rb;
    float ca, cb, c0;
    // columns: coordinates [D][col_ld], exponent term cbeta [col_ld];
    //   A_COL: cw = V [D+1][col_ld], the weight w and its moments w xhat;
    //   A_FCOL: cw = A [D][col_ld], cgam = Gamma [col_ld]
    const float* cols;
    const float* cbeta;
    const float* cw;
    const float* cgam;
    int col_ld;
    int n_cols8, cols_per_split, splits;
    int n_hi;    // row blocks with `splits` splits; the others have splits - 1 of cps_lo columns
    int cps_lo;
    float* part;
    int part_ld;
    unsigned* counters;
    int n_rb;
    int pre_ok;  // row/column coordinates were written before the previous launch
    // epilogue (see adj_epilogue)
    int epi;
    float sig, eps, log2a;
    float* xbar;
    float* xbarp;
    float* ybar;
    float* lbbar;
    float* w_out;
    float* beta_out;
    float* gam_out;
    const float* h0;
    const float* h1;
    const float* geo;
    const float* w_in;
    const float* A;
    unsigned* status;
    long long spin_limit;
};

struct AdjLaunch {
    AdjArgs seg[2];
    int ctas0;
};

__device__ __forceinline__ void adj_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void adj_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <int D>
__device__ __forceinline__ constexpr int sym_idx(int k, int l) {
    return k * D - k * (k - 1) / 2 + (l - k);
}

constexpr float kTwoLn2 = 1.3862943611198906f;

// The staged column values of the next reverse pass: V = w [1, xhat].
template <int D>
__device__ __forceinline__ void write_v(float* V, size_t ld, int i, float w, const float* xh) {
    V[i] = w;
#pragma unroll
    for (int k = 0; k < D; ++k) V[(1 + k) * ld + i] = w * xh[k];
}

template <int D, int KIND>
__device__ void adj_epilogue(const AdjArgs& a, int i, const float* acc) {
    if (i >= a.n_rows) return;
    bool ok = true;
    const size_t ld = (size_t)a.row_ld;
    float xh[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xh[k] = a.rows[k * ld + i];
    const float s2 = 2.0f * a.sig;
    if constexpr (KIND == A_COL) {
        const float W = acc[0];
        if (a.epi == E_FREV) {
            const float gb = -W;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float v = a.ybar[k * ld + i] + s2 * (xh[k] * W - acc[1 + k]) - s2 * gb * a.geo[k * ld + i];
                a.ybar[k * ld + i] = v;
                ok &= finitef(v);
            }
            const float l = a.lbbar[i] - a.eps * W;
            a.lbbar[i] = l;
            ok &= finitef(l);
            write_v<D>(a.w_out, ld, i, gb, xh);
            a.beta_out[i] = a.h0[i] - a.h1[i];
        } else if (a.epi == E_GREV) {
            const float fb = -W;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                float v = a.xbar[k * ld + i] + s2 * (xh[k] * W - acc[1 + k]);
                if (a.geo) v -= s2 * fb * a.geo[k * ld + i];
                a.xbar[k * ld + i] = v;
                ok &= finitef(v);
            }
            if (a.w_out) write_v<D>(a.w_out, ld, i, fb, xh);
        } else {  // E_PREV
            const float pt = 2.0f * a.w_in[i];  // row 0 of the staged V: pbar^t / 2
            const float pm = 0.5f * pt - W;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float v =
                    a.xbarp[k * ld + i] + s2 * (xh[k] * W - acc[1 + k]) - a.sig * pt * a.geo[k * ld + i];
                a.xbarp[k * ld + i] = v;
                ok &= finitef(v);
            }
            if (a.w_out) {
                write_v<D>(a.w_out, ld, i, 0.5f * pm, xh);
                a.beta_out[i] = 2.0f * a.h0[i] - a.log2a - a.h1[i];
            }
        }
    } else if constexpr (KIND == A_MOM) {
        const float inv = 1.0f / acc[0];
        float eb[D], Ai[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            eb[k] = acc[1 + k] * inv;
            Ai[k] = a.A[k * ld + i];
        }
        float* xb = (a.epi == E_MOM_CROSS) ? a.xbar : a.xbarp;
        float gam = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            float ca = 0.f;
#pragma unroll
            for (int l = 0; l < D; ++l) {
                const int q = k <= l ? sym_idx<D>(k, l) : sym_idx<D>(l, k);
                const float c = acc[1 + D + q] * inv - eb[k] * eb[l];
                ca = fmaf(c, Ai[l], ca);
            }
            const float v = xb[k * ld + i] + kTwoLn2 * ca;
            xb[k * ld + i] = v;
            ok &= finitef(v);
            gam = fmaf(Ai[k], xh[k] + eb[k], gam);
        }
        a.gam_out[i] = gam;
        ok &= finitef(gam);
        if (a.epi == E_MOM_SELF) a.beta_out[i] = a.ca * a.ra[i] + (a.rb ? a.cb * a.rb[i] : 0.f) + a.c0;
    } else {  // A_FCOL
        const float W1 = acc[0];
        if (a.epi == E_FCOL_CROSS) {
            const float gb = a.sig * W1 / a.eps;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                float v = a.ybar[k * ld + i] + acc[1 + k] - kTwoLn2 * acc[1 + D + k];
                if (a.geo) v -= s2 * gb * a.geo[k * ld + i];
                a.ybar[k * ld + i] = v;
                ok &= finitef(v);
            }
            const float l = a.lbbar[i] + a.sig * W1;
            a.lbbar[i] = l;
            ok &= finitef(l);
            write_v<D>(a.w_out, ld, i, gb, xh);
            a.beta_out[i] = a.h0[i] - a.h1[i];
        } else {  // E_FCOL_SELF
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float v = a.xbarp[k * ld + i] + acc[1 + k] - kTwoLn2 * acc[1 + D + k];
                a.xbarp[k * ld + i] = v;
                ok &= finitef(v);
            }
            if (a.w_out) {
                write_v<D>(a.w_out, ld, i, 0.5f * a.sig * W1 / a.eps, xh);
                a.beta_out[i] = 2.0f * a.h0[i] - a.log2a - a.h1[i];
            }
        }
    }
    if (!ok) raise_status(a.status, kDevNonfinite);
}

// One 8-column chunk of a tile for the R rows of this lane.
template <int D, int KIND>
__device__ __forceinline__ void adj_chunk(const float* __restrict__ st, int j, const float (&X2)[AdjTraits<D, KIND>::R][D],
                                          const float (&Xr)[AdjTraits<D, KIND>::R][D],
                                          const float (&al)[AdjTraits<D, KIND>::R],
                                          float2 (&acc)[AdjTraits<D, KIND>::R][AdjTraits<D, KIND>::NACC]) {
    using TR = AdjTraits<D, KIND>;
    constexpr int R = TR::R, NC = TR::NC;
    float c[NC][8];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float4 v0 = *reinterpret_cast<const float4*>(st + k * kATile + j);
        const float4 v1 = *reinterpret_cast<const float4*>(st + k * kATile + j + 4);
        c[k][0] = v0.x; c[k][1] = v0.y; c[k][2] = v0.z; c[k][3] = v0.w;
        c[k][4] = v1.x; c[k][5] = v1.y; c[k][6] = v1.z; c[k][7] = v1.w;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 al2 = make_float2(al[r], al[r]);
        float2 e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float2 w = add2(make_float2(c[D][2 * q], c[D][2 * q + 1]), al2);
#pragma unroll
            for (int k = 0; k < D; ++k)
                w = fma2(make_float2(X2[r][k], X2[r][k]), make_float2(c[k][2 * q], c[k][2 * q + 1]), w);
            e[q] = make_float2(ex2(w.x), ex2(w.y));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (KIND == A_COL) {  // staged [D coords][beta][V: w, w xhat]
#pragma unroll
                for (int k = 0; k <= D; ++k)
                    acc[r][k] = fma2(e[q], make_float2(c[D + 1 + k][2 * q], c[D + 1 + k][2 * q + 1]), acc[r][k]);
            } else if constexpr (KIND == A_MOM) {
                float2 dk[D], ek[D];
                acc[r][0] = add2(acc[r][0], e[q]);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    dk[k] = sub2(make_float2(c[k][2 * q], c[k][2 * q + 1]), make_float2(Xr[r][k], Xr[r][k]));
                    ek[k] = mul2(e[q], dk[k]);
                    acc[r][1 + k] = add2(acc[r][1 + k], ek[k]);
                }
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                    for (int l = k; l < D; ++l)
                        acc[r][1 + D + sym_idx<D>(k, l)] = fma2(ek[k], dk[l], acc[r][1 + D + sym_idx<D>(k, l)]);
            } else {  // A_FCOL: staged [D coords][beta][D A][Gamma]
                float2 u = mul2(make_float2(c[D + 1][2 * q], c[D + 1][2 * q + 1]), make_float2(Xr[r][0], Xr[r][0]));
#pragma unroll
                for (int k = 1; k < D; ++k)
                    u = fma2(make_float2(c[D + 1 + k][2 * q], c[D + 1 + k][2 * q + 1]), make_float2(Xr[r][k], Xr[r][k]), u);
                u = sub2(u, make_float2(c[2 * D + 1][2 * q], c[2 * D + 1][2 * q + 1]));
                const float2 eu = mul2(e[q], u);
                acc[r][0] = add2(acc[r][0], eu);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    acc[r][1 + k] = fma2(e[q], make_float2(c[D + 1 + k][2 * q], c[D + 1 + k][2 * q + 1]), acc[r][1 + k]);
                    acc[r][1 + D + k] = fma2(eu, sub2(make_float2(Xr[r][k], Xr[r][k]), make_float2(c[k][2 * q], c[k][2 * q + 1])),
                                             acc[r][1 + D + k]);
                }
            }
        }
    }
}

template <int D, int KIND>
__global__ void __launch_bounds__(kAThreads) adj_kernel(const __grid_constant__ AdjLaunch L) {
    using TR = AdjTraits<D, KIND>;
    constexpr int R = TR::R, NC = TR::NC, NACC = TR::NACC, RB = 32 * R;
    __shared__ __align__(128) float sm[2][NC * kATile];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red[kAWarps][NACC][RB];
    __shared__ int s_last;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int segi = ((int)blockIdx.x >= L.ctas0) ? 1 : 0;
    const AdjArgs& a = segi ? L.seg[1] : L.seg[0];
    const int lb = (int)blockIdx.x - (segi ? L.ctas0 : 0);
    // this CTA's row block, split index, the row block's split count and its
    // columns (a plan may give some row blocks one split fewer)
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
    if (!a.pre_ok) adj_dep_wait();

    // rows and their exponent terms come from the forward record (constant
    // during the reverse sweep)
    float X2[R][D], Xr[R][D], al[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row0 + r * 32 + lane;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float v = a.rows[(size_t)k * a.row_ld + i];
            X2[r][k] = 2.0f * v;
            Xr[r][k] = v;
        }
        al[r] = a.ca * a.ra[i] + (a.rb ? a.cb * a.rb[i] : 0.f) + a.c0;
    }
    float2 acc[R][NACC];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < NACC; ++k) acc[r][k] = make_float2(0.f, 0.f);

    const int c0 = sp * cps;
    const int c1 = min(c0 + cps, a.n_cols8);
    const int n_tiles = c1 > c0 ? (c1 - c0 + kATile - 1) / kATile : 0;
    __syncthreads();

    auto issue_coords = [&](int t, int stg) {
        const int tc = c0 + t * kATile;
        const unsigned bytes = (unsigned)min(kATile, c1 - tc) * 4u;
        mbar_arrive_expect_tx(&bar[stg], bytes * NC);
#pragma unroll
        for (int k = 0; k < D; ++k) bulk_g2s(&sm[stg][k * kATile], a.cols + (size_t)k * a.col_ld + tc, bytes, &bar[stg]);
    };
    auto issue_rest = [&](int t, int stg) {
        const int tc = c0 + t * kATile;
        const unsigned bytes = (unsigned)min(kATile, c1 - tc) * 4u;
        bulk_g2s(&sm[stg][D * kATile], a.cbeta + tc, bytes, &bar[stg]);
        if constexpr (KIND == A_COL) {
#pragma unroll
            for (int k = 0; k <= D; ++k)
                bulk_g2s(&sm[stg][(D + 1 + k) * kATile], a.cw + (size_t)k * a.col_ld + tc, bytes, &bar[stg]);
        } else if constexpr (KIND == A_FCOL) {
#pragma unroll
            for (int k = 0; k < D; ++k)
                bulk_g2s(&sm[stg][(D + 1 + k) * kATile], a.cw + (size_t)k * a.col_ld + tc, bytes, &bar[stg]);
            bulk_g2s(&sm[stg][(2 * D + 1) * kATile], a.cgam + tc, bytes, &bar[stg]);
        }
    };

    if (threadIdx.x == 0 && n_tiles > 0) issue_coords(0, 0);
    if (a.pre_ok) adj_dep_wait();
    adj_dep_launch();
    if (threadIdx.x == 0 && n_tiles > 0) issue_rest(0, 0);
    int bad_tile = -1;
    for (int t = 0; t < n_tiles; ++t) {
        const int stg = t & 1;
        if (threadIdx.x == 0 && t + 1 < n_tiles) {
            issue_coords(t + 1, stg ^ 1);
            issue_rest(t + 1, stg ^ 1);
        }
        const bool ok = mbar_wait_bounded(&bar[stg], (unsigned)((t >> 1) & 1), a.spin_limit);
        if (__syncthreads_or(!ok)) {
            bad_tile = t;
            break;
        }
        const int nc = min(kATile, c1 - (c0 + t * kATile));
        const int per = ((nc / 8 + kAWarps - 1) / kAWarps) * 8;
        const int jb = min(nc, warp * per), je = min(nc, jb + per);
#pragma unroll 1
        for (int j = jb; j < je; j += 8) adj_chunk<D, KIND>(sm[stg], j, X2, Xr, al, acc);
        __syncthreads();
    }
    if (bad_tile >= 0) {
        // a tile never arrived: record it, drain the copies in flight
        // (bounded) and fall through (the status marks the result invalid)
        if (threadIdx.x == 0) {
            raise_status(a.status, kDevTimeout);
            const long long drain = a.spin_limit > (1LL << 20) ? a.spin_limit : (1LL << 20);
            mbar_wait_bounded(&bar[bad_tile & 1], (unsigned)((bad_tile >> 1) & 1), drain);
            if (bad_tile + 1 < n_tiles)
                mbar_wait_bounded(&bar[(bad_tile + 1) & 1], (unsigned)(((bad_tile + 1) >> 1) & 1), drain);
        }
        __syncthreads();
    }

    // ---- reduce the 4 warps' partials of each row ---------------------------
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < NACC; ++k) red[warp][k][r * 32 + lane] = acc[r][k].x + acc[r][k].y;
    __syncthreads();
    for (int q = threadIdx.x; q < RB; q += kAThreads) {
        float tot[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) {
            float v = red[0][k][q];
#pragma unroll
            for (int w = 1; w < kAWarps; ++w) v += red[w][k][q];
            tot[k] = v;
        }
        const int i = row0 + q;
        if (ns == 1) {
            adj_epilogue<D, KIND>(a, i, tot);
        } else {
            float* P = a.part + (size_t)sp * a.part_ld + i;
            const size_t cs = (size_t)a.splits * a.part_ld;
#pragma unroll
            for (int k = 0; k < NACC; ++k) P[k * cs] = tot[k];
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
    for (int q = threadIdx.x; q < RB; q += kAThreads) {
        const int i = row0 + q;
        float tot[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) tot[k] = 0.f;
        // splits in groups of 8, all loads of a group in flight together
        for (int p0 = 0; p0 < ns; p0 += 8) {
            float v[8][NACC];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool live = p0 + u < ns;
                const float* P = a.part + (size_t)(live ? p0 + u : 0) * a.part_ld + i;
#pragma unroll
                for (int k = 0; k < NACC; ++k) v[u][k] = live ? ld_cg(P + k * cs) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int k = 0; k < NACC; ++k) tot[k] += v[u][k];
        }
        adj_epilogue<D, KIND>(a, i, tot);
    }
    if (threadIdx.x == 0) a.counters[rb] = 0u;  // ready for the next launch
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int D, int KIND>
static int adj_occupancy() {
    static int occ = 0;
    if (occ == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, adj_kernel<D, KIND>, kAThreads, 0) != cudaSuccess ||
            v < 1) {
            cudaGetLastError();
            v = 1;
        }
        occ = v;
    }
    return occ;
}

template <int D, int KIND>
static cudaError_t adj_launch_t(const AdjLaunch& L, int n_ctas, cudaStream_t st, int* occ) {
    if (occ) {
        *occ = adj_occupancy<D, KIND>();
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)n_ctas);
    cfg.blockDim = dim3(kAThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, adj_kernel<D, KIND>, L);
}

template <int D>
static cudaError_t adj_launch_k(int kind, const AdjLaunch& L, int n, cudaStream_t st, int* occ) {
    switch (kind) {
        case A_COL: return adj_launch_t<D, A_COL>(L, n, st, occ);
        case A_MOM: return adj_launch_t<D, A_MOM>(L, n, st, occ);
        case A_FCOL: return adj_launch_t<D, A_FCOL>(L, n, st, occ);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t adj_launch(int d, int kind, const AdjLaunch& L, int n, cudaStream_t st, int* occ) {
    switch (d) {
        case 1: return adj_launch_k<1>(kind, L, n, st, occ);
        case 2: return adj_launch_k<2>(kind, L, n, st, occ);
        case 3: return adj_launch_k<3>(kind, L, n, st, occ);
    }
    return cudaErrorInvalidValue;
}

static int adj_rows_per_cta(int kind) { return kind == A_COL ? 128 : 64; }
static int adj_nacc(int kind, int d) {
    return kind == A_COL ? d + 1 : (kind == A_MOM ? 1 + d + d * (d + 1) / 2 : 1 + 2 * d);
}

// Exact one-wave plans (fill_plan) for the reverse kernel (build flag
// -DCOV_ADJ_FILL=0 keeps the uniform plan).
#ifndef COV_ADJ_FILL
#define COV_ADJ_FILL 1
#endif
// Fewest 8-column units per split the re-plan may leave (build flag; default one tile).
#ifndef COV_ADJ_FILL_MIN_UNITS
#define COV_ADJ_FILL_MIN_UNITS (kATile / 8)
#endif

// Uniform split plan; when it is one wave that already fills at least half
// of `slots`, re-planned to fill them exactly (as the forward kernel does).
static void adj_plan(AdjArgs& a, int n_cols, int RB, int slots, unsigned* counters) {
    const SplitPlan pl = plan_splits(a.n_rows, n_cols, RB, slots);
    a.n_cols8 = (int)round_up((size_t)n_cols, 8);
    a.cols_per_split = pl.cols_per_split;
    a.splits = pl.splits;
    a.n_rb = pl.n_rb;
    a.n_hi = pl.n_rb;
    a.cps_lo = pl.cols_per_split;
    a.part_ld = pl.n_rb * RB;
    a.counters = counters;
    const long long ctas = (long long)a.n_rb * a.splits;
    if (COV_ADJ_FILL && ctas <= slots && 2 * ctas >= slots && slots > a.n_rb)
        fill_plan(a, n_cols, slots, 8, COV_ADJ_FILL_MIN_UNITS);
}

static int adj_ctas(const AdjArgs& a) { return a.n_hi * a.splits + (a.n_rb - a.n_hi) * (a.splits - 1); }

// One or two passes of one kind in a single grid (as run_pairs in field.cu).
static cov_status run_adj(cov_ctx* ctx, int d, int kind, AdjArgs* seg, const int* n_cols, int nseg,
                          unsigned* counters, int cnt_ld, cudaStream_t st) {
    const int RB = adj_rows_per_cta(kind);
    int occ = 1;
    adj_launch(d, kind, AdjLaunch{}, 0, st, &occ);
    const int slots = std::max(1, std::min(ctx->num_sms * std::min(occ, ctx->ctas_per_sm), kAMaxSlots));
    AdjLaunch L{};
    if (nseg == 1) {
        adj_plan(seg[0], n_cols[0], RB, slots, counters);
        L.seg[0] = seg[0];
        L.seg[1] = seg[0];
        L.ctas0 = adj_ctas(seg[0]);
    } else {
        const double w0 = (double)seg[0].n_rows * n_cols[0], w1 = (double)seg[1].n_rows * n_cols[1];
        int s0 = (int)llround(slots * w0 / (w0 + w1));
        s0 = std::max(1, std::min(s0, slots - 1));
        const int s1 = std::max(1, slots - s0);
        adj_plan(seg[0], n_cols[0], RB, s0, counters);
        adj_plan(seg[1], n_cols[1], RB, s1, counters + cnt_ld);
        seg[1].part = seg[0].part + (size_t)adj_nacc(kind, d) * seg[0].splits * seg[0].part_ld;
        L.seg[0] = seg[0];
        L.seg[1] = seg[1];
        L.ctas0 = adj_ctas(seg[0]);
    }
    const int total = L.ctas0 + (nseg == 2 ? adj_ctas(seg[1]) : 0);
    const cudaError_t e = adj_launch(d, kind, L, total, st, nullptr);
    return cuda_failed(ctx, e) ? COV_ERR_CUDA : COV_OK;
}

struct VjpBufs {
    float *A, *B;          // [d][Tp]: 2 abar, -2 abar (padding 0)
    float *xbar, *xbarp;   // [d][Tp]: x adjoint of the cross/g-f chain and of the self/p chain
    float* ybar;           // [d][Mp]
    float* lbbar;          // [Mp]: d/d log b (normalised)
    float *gw, *gbeta;     // g-step columns: V = gbar [1, yhat] [d+1][Mp], exponent terms [Mp]
    float* fw;             // f-step columns: V = fbar [1, xhat] [d+1][Tp]
    float *pw[2], *pbeta[2];  // p-step columns: V = pbar/2 [1, xhat] [d+1][Tp], terms [Tp]; ping-pong
    float *gam_c, *gam_s, *sbeta;  // [Tp]
    float* part;
    unsigned* counters;    // [2][cnt_ld]
    int cnt_ld;
};

static VjpBufs carve_vjp(Carver& cv, int d, int Tp, int Mp) {
    VjpBufs v{};
    v.A = cv.take<float>((size_t)d * Tp);
    v.B = cv.take<float>((size_t)d * Tp);
    v.xbar = cv.take<float>((size_t)d * Tp);
    v.xbarp = cv.take<float>((size_t)d * Tp);
    v.ybar = cv.take<float>((size_t)d * Mp);
    v.lbbar = cv.take<float>(Mp);
    v.gw = cv.take<float>((size_t)(d + 1) * Mp);
    v.gbeta = cv.take<float>(Mp);
    v.fw = cv.take<float>((size_t)(d + 1) * Tp);
    for (int q = 0; q < 2; ++q) {
        v.pw[q] = cv.take<float>((size_t)(d + 1) * Tp);
        v.pbeta[q] = cv.take<float>(Tp);
    }
    v.gam_c = cv.take<float>(Tp);
    v.gam_s = cv.take<float>(Tp);
    v.sbeta = cv.take<float>(Tp);
    v.cnt_ld = std::max(Tp, Mp) / 32 + 1;
    v.counters = cv.take<unsigned>((size_t)2 * v.cnt_ld);
    const int nacc = std::max(adj_nacc(A_MOM, d), adj_nacc(A_FCOL, d));
    v.part = cv.take<float>((size_t)nacc * (kAPartRows + Tp + Mp));
    return v;
}

__global__ void vjp_init_kernel(const float* __restrict__ abar, int abar_ld, int T, int M, int d, int Tp, int Mp,
                                VjpBufs v, unsigned* status) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Tp) {
        bool ok = true;
        for (int k = 0; k < d; ++k) {
            const float av = i < T ? 2.0f * abar[(size_t)i * abar_ld + k] : 0.f;
            ok &= finitef(av);
            v.A[(size_t)k * Tp + i] = av;
            v.B[(size_t)k * Tp + i] = -av;
            v.xbar[(size_t)k * Tp + i] = 0.f;
            v.xbarp[(size_t)k * Tp + i] = 0.f;
        }
        if (!ok) raise_status(status, kDevNonfinite);
        for (int k = 0; k <= d; ++k) {
            v.fw[(size_t)k * Tp + i] = 0.f;
            v.pw[0][(size_t)k * Tp + i] = 0.f;
            v.pw[1][(size_t)k * Tp + i] = 0.f;
        }
        v.pbeta[0][i] = kPadH;
        v.pbeta[1][i] = kPadH;
        v.gam_c[i] = 0.f;
        v.gam_s[i] = 0.f;
        v.sbeta[i] = kPadH;
    }
    if (i < Mp) {
        for (int k = 0; k < d; ++k) v.ybar[(size_t)k * Mp + i] = 0.f;
        v.lbbar[i] = 0.f;
        for (int k = 0; k <= d; ++k) v.gw[(size_t)k * Mp + i] = 0.f;
        v.gbeta[i] = kPadH;
    }
    if (i < 2 * v.cnt_ld) v.counters[i] = 0u;
}

// Outputs in the caller's layout; the weight adjoint needs sum_j lbbar_j
// (one CTA).
__global__ void __launch_bounds__(1024) vjp_finish_kernel(VjpBufs v, int T, int M, int d, int Tp, int Mp,
                                                          const float* __restrict__ b, const float* __restrict__ scal,
                                                          float* __restrict__ xbar, int xbar_ld,
                                                          float* __restrict__ ybar, float* __restrict__ bbar,
                                                          int accumulate, unsigned* status) {
    pdl_prologue();
    __shared__ double sh[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    bool ok = true;
    for (int i = tid; i < T; i += nt)
        for (int k = 0; k < d; ++k) {
            const float x = v.xbar[(size_t)k * Tp + i] + v.xbarp[(size_t)k * Tp + i];
            xbar[(size_t)i * xbar_ld + k] = x;
            ok &= finitef(x);
        }
    for (int j = tid; j < M; j += nt)
        for (int k = 0; k < d; ++k) {
            const float y = v.ybar[(size_t)k * Mp + j];
            ybar[(size_t)j * d + k] = accumulate ? ybar[(size_t)j * d + k] + y : y;
        }
    if (b && bbar) {
        double s = 0.0;
        for (int j = tid; j < M; j += nt) s += v.lbbar[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((tid & 31) == 0) sh[tid >> 5] = s;
        __syncthreads();
        if (tid < 32) {
            double t = tid < (nt >> 5) ? sh[tid] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (tid == 0) sh[0] = t;
        }
        __syncthreads();
        // scal[8] = 1 / sum b
        const float mean = (float)(sh[0] * (double)scal[8]);
        for (int j = tid; j < M; j += nt) {
            const float g = v.lbbar[j] / b[j] - mean;
            bbar[j] = accumulate ? bbar[j] + g : g;
            ok &= finitef(g);
        }
    }
    if (!ok) raise_status(status, kDevNonfinite);
}

size_t sinkhorn_vjp_bytes(int T, int M, int d, int n_iter) {
    return round_up(sinkhorn_tape_bytes(T, M, d, n_iter), 256) + sinkhorn_vjp_bytes_given(T, M, d);
}

size_t sinkhorn_vjp_bytes_given(int T, int M, int d) {
    Carver cv(nullptr);
    const int Tp = (int)round_up((size_t)T, 1024), Mp = (int)round_up((size_t)M, 1024);
    carve_vjp(cv, d, Tp, Mp);
    return round_up(cv.off, 256);
}

cov_status sinkhorn_vjp_ws(cov_ctx* ctx, void* ws, size_t ws_bytes, const float* x, int x_ld, int T,
                           const float* y, const float* b, int M, int d, float eps, int n_iter,
                           const float* scal_given, const float* abar, int abar_ld, float* xbar, int xbar_ld,
                           float* ybar, float* bbar, int accumulate, cudaStream_t stream,
                           const SkTape* given_tape) {
    if (!ctx || !x || !y || !abar || !xbar || !ybar || T < 1 || M < 1 || d < 1 || n_iter < 0 || x_ld < d ||
        abar_ld < d || xbar_ld < d || !(eps > 0.f) || !isfinite(eps))
        return COV_ERR_INVALID_ARG;
    if (d > 3) return COV_ERR_UNSUPPORTED;
    SkTape tp{};
    size_t used = 0;
    cov_status r = COV_OK;
    if (given_tape) {
        tp = *given_tape;
        if (tp.n_iter != n_iter || tp.T != T || tp.M != M || tp.d != d || tp.eps != eps) return COV_ERR_INVALID_ARG;
    } else {
        r = sinkhorn_tape_ws(ctx, ws, ws_bytes, x, x_ld, T, y, b, M, d, eps, n_iter, scal_given, &tp, &used,
                             stream);
        if (r != COV_OK) return r;
    }
    Carver cv(ws);
    cv.off = used;
    VjpBufs v = carve_vjp(cv, d, tp.Tp, tp.Mp);
    if (cv.off > ws_bytes) return COV_ERR_WORKSPACE;
    const int n = n_iter, Tp = tp.Tp, Mp = tp.Mp;
    const int np = std::max(std::max(Tp, Mp), 2 * v.cnt_ld);
    launch_pdl(vjp_init_kernel, dim3((np + 255) / 256), dim3(256), 0, stream, abar, abar_ld, T, M, d, Tp, Mp, v, ctx->status);
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;

    auto hx = [&](int t) { return tp.hx + (size_t)t * Tp; };
    auto hy = [&](int t) { return tp.hy + (size_t)t * Mp; };
    auto hp = [&](int t) { return tp.hp + (size_t)t * Tp; };
    AdjArgs base{};
    base.status = ctx->status;
    base.spin_limit = ctx->spin_limit;
    base.part = v.part;
    base.pre_ok = 1;
    base.sig = tp.sigma;
    base.eps = eps;
    base.log2a = tp.log2a;
    base.xbar = v.xbar;
    base.xbarp = v.xbarp;
    base.ybar = v.ybar;
    base.lbbar = v.lbbar;
    base.ca = 1.f;
    auto rows_x = [&](AdjArgs& a) { a.rows = tp.xs; a.row_ld = Tp; a.n_rows = T; };
    auto rows_y = [&](AdjArgs& a) { a.rows = tp.ys; a.row_ld = Mp; a.n_rows = M; };
    auto cols_x = [&](AdjArgs& a) { a.cols = tp.xs; a.col_ld = Tp; };
    auto cols_y = [&](AdjArgs& a) { a.cols = tp.ys; a.col_ld = Mp; };

    // ---- the field: covariance row passes, then column passes ----------------
    {
        AdjArgs s[2] = {base, base};
        rows_x(s[0]); cols_y(s[0]);
        s[0].ra = hx(n); s[0].c0 = -tp.log2a; s[0].cbeta = hy(n);
        s[0].epi = E_MOM_CROSS; s[0].A = v.A; s[0].gam_out = v.gam_c;
        rows_x(s[1]); cols_x(s[1]);
        s[1].ra = hp(n + 1); s[1].ca = 2.f; s[1].rb = hp(n); s[1].cb = -1.f; s[1].c0 = -tp.log2a;
        s[1].cbeta = hp(n);
        s[1].epi = E_MOM_SELF; s[1].A = v.B; s[1].gam_out = v.gam_s; s[1].beta_out = v.sbeta;
        const int nc[2] = {M, T};
        r = run_adj(ctx, d, A_MOM, s, nc, 2, v.counters, v.cnt_ld, stream);
        if (r != COV_OK) return r;
    }
    {
        AdjArgs s[2] = {base, base};
        rows_y(s[0]); cols_x(s[0]);
        s[0].ra = hy(n); s[0].c0 = -tp.log2a; s[0].cbeta = hx(n); s[0].cw = v.A; s[0].cgam = v.gam_c;
        s[0].epi = E_FCOL_CROSS; s[0].w_out = v.gw; s[0].beta_out = v.gbeta; s[0].h0 = hy(n); s[0].h1 = tp.lb;
        s[0].geo = n >= 1 ? tp.Dg + (size_t)n * d * Mp : nullptr;
        rows_x(s[1]); cols_x(s[1]);
        s[1].ra = hp(n); s[1].cbeta = v.sbeta; s[1].cw = v.B; s[1].cgam = v.gam_s;
        s[1].epi = E_FCOL_SELF;
        if (n >= 1) {
            s[1].w_out = v.pw[0]; s[1].beta_out = v.pbeta[0]; s[1].h0 = hp(n); s[1].h1 = hp(n - 1);
        }
        const int nc[2] = {T, T};
        r = run_adj(ctx, d, A_FCOL, s, nc, 2, v.counters, v.cnt_ld, stream);
        if (r != COV_OK) return r;
    }
    // ---- reverse iterations t = n..1 -----------------------------------------
    int cur = 0;
    for (int t = n; t >= 1; --t) {
        if (t < n) {  // f-step of iteration t (fbar^n = 0: nothing at t = n)
            AdjArgs a = base;
            rows_y(a); cols_x(a);
            a.ra = hy(t); a.c0 = -tp.log2a; a.cbeta = hx(t); a.cw = v.fw;
            a.epi = E_FREV; a.w_out = v.gw; a.beta_out = v.gbeta; a.h0 = hy(t); a.h1 = tp.lb;
            a.geo = tp.Dg + (size_t)t * d * Mp;
            const int nc[1] = {T};
            r = run_adj(ctx, d, A_COL, &a, nc, 1, v.counters, v.cnt_ld, stream);
            if (r != COV_OK) return r;
        }
        AdjArgs s[2] = {base, base};
        rows_x(s[0]); cols_y(s[0]);  // g-step of iteration t
        s[0].ra = hx(t - 1); s[0].cbeta = v.gbeta; s[0].cw = v.gw;
        s[0].epi = E_GREV;
        if (t >= 2) {
            s[0].w_out = v.fw;
            s[0].geo = tp.Df + (size_t)(t - 1) * d * Tp;
        }
        rows_x(s[1]); cols_x(s[1]);  // p-step of iteration t
        s[1].ra = hp(t - 1); s[1].cbeta = v.pbeta[cur]; s[1].cw = v.pw[cur];
        s[1].epi = E_PREV; s[1].w_in = v.pw[cur]; s[1].geo = tp.Dp + (size_t)t * d * Tp;
        if (t >= 2) {
            s[1].w_out = v.pw[cur ^ 1]; s[1].beta_out = v.pbeta[cur ^ 1]; s[1].h0 = hp(t - 1); s[1].h1 = hp(t - 2);
        }
        const int nc[2] = {M, T};
        r = run_adj(ctx, d, A_COL, s, nc, 2, v.counters, v.cnt_ld, stream);
        if (r != COV_OK) return r;
        cur ^= 1;
    }
    launch_pdl(vjp_finish_kernel, dim3(1), dim3(1024), 0, stream, v, T, M, d, Tp, Mp, b, tp.scal, xbar, xbar_ld, ybar, bbar,
                                              accumulate, ctx->status);
    if (cuda_failed(ctx, cudaGetLastError())) return COV_ERR_CUDA;
    return COV_OK;
}

}  // namespace cov

extern "C" size_t cov_workspace_size_vjp(int T, int M, int d, int n_iter) {
    if (T < 1 || M < 1 || d < 1 || d > 3 || n_iter < 0) return 0;
    return cov::sinkhorn_vjp_bytes(T, M, d, n_iter) + 4096;
}

extern "C" cov_status cov_field_sinkhorn_vjp(cov_ctx* ctx, const float* x, int T, const float* y, const float* b,
                                             int M, int d, float eps, int n_iter, const float* abar, float* xbar,
                                             float* ybar, float* bbar, cov_stream_t stream) {
    if (!ctx) return COV_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return COV_ERR_CUDA;
    cov::clobber_ws_caches(ctx);  // the workspace scratch overwrites cov_solve's caches
    return cov::sinkhorn_vjp_ws(ctx, ctx->ws, ctx->ws_bytes, x, d, T, y, b, M, d, eps, n_iter, nullptr, abar, d,
                                xbar, d, ybar, b ? bbar : nullptr, 0, (cudaStream_t)stream);
}
