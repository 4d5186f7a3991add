/*
 * cov_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see the
 * header for who may load it).  Every function below restates one step of
 * the method of Sun, Kwon, Murphey, "Scalable Coverage Trajectory Synthesis
 * on GPUs as Statistical Inference" (arXiv 2511.11514), in the paper's order
 * and notation, with plain loops and no blocking, fusion or reordering.
 * Where the paper is silent the reading used is stated next to the code.
 *
 * Row loops carry an OpenMP "parallel for": rows are independent by
 * definition, so this changes no arithmetic.
 */
#include "cov_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* log-sum-exp of z[0..n-1], max-subtracted. */
static double lse(const double* z, int n) {
    double m = -INFINITY;
    for (int k = 0; k < n; ++k)
        if (z[k] > m) m = z[k];
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += exp(z[k] - m);
    return m + log(s);
}

/* c(x, y) = |x - y|^2: the squared-norm cost of Sec. II-B (Eq. 5). */
static double sqdist(const double* u, const double* v, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = u[k] - v[k];
        s += t * t;
    }
    return s;
}

static int row_index(const int* rows, int r) { return rows ? rows[r] : r; }

/* ------------------------------------------------------------------------
 * Reference distribution q (Sec. II-A): an isotropic Gaussian mixture
 *   q(x) = sum_k w_k N(x; mu_k, sigma_k^2 I).
 * ---------------------------------------------------------------------- */
static void gmm_log_terms(const double* x, int d, int K, const double* w,
                          const double* mu, const double* sigma, double* t) {
    const double log2pi = log(2.0 * M_PI);
    for (int k = 0; k < K; ++k) {
        double s2 = sigma[k] * sigma[k];
        t[k] = log(w[k]) - 0.5 * d * (log2pi + log(s2)) -
               sqdist(x, mu + (size_t)k * d, d) / (2.0 * s2);
    }
}

double orc_gmm_logpdf(const double* x, int d, int K, const double* w,
                      const double* mu, const double* sigma) {
    double* t = (double*)malloc(sizeof(double) * K);
    gmm_log_terms(x, d, K, w, mu, sigma, t);
    double r = lse(t, K);
    free(t);
    return r;
}

/* Score grad log q(x) = sum_k r_k(x) (mu_k - x) / sigma_k^2, with the
 * responsibilities r_k the softmax of the component log terms.  Only the
 * score is needed by Eq. 4 (Sec. II-B, last paragraph). */
void orc_gmm_score(const double* x, int T, int d, int K, const double* w,
                   const double* mu, const double* sigma, double* score) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < T; ++i) {
        double* t = (double*)malloc(sizeof(double) * K);
        const double* xi = x + (size_t)i * d;
        gmm_log_terms(xi, d, K, w, mu, sigma, t);
        double L = lse(t, K);
        for (int c = 0; c < d; ++c) score[(size_t)i * d + c] = 0.0;
        for (int k = 0; k < K; ++k) {
            double r = exp(t[k] - L);
            double s2 = sigma[k] * sigma[k];
            for (int c = 0; c < d; ++c)
                score[(size_t)i * d + c] += r * (mu[(size_t)k * d + c] - xi[c]) / s2;
        }
        free(t);
    }
}

/* ------------------------------------------------------------------------
 * Stein variational gradient field, Eq. 4:
 *   g(x_i) = 1/T sum_j [ k(x_j, x_i) grad log q(x_j) + grad_{x_j} k(x_j, x_i) ]
 * Reading of the radial basis kernel: k(x, x') = exp(-|x - x'|^2 / (2 h^2)),
 * so grad_{x_j} k(x_j, x_i) = k(x_j, x_i) (x_i - x_j) / h^2.  The j = i term
 * is part of the sum.
 * ---------------------------------------------------------------------- */
void orc_svgd_field(const double* x, int T, int d, const double* score,
                    double h, const int* rows, int n_rows, double* out) {
    int nr = rows ? n_rows : T;
    double h2 = h * h;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nr; ++r) {
        int i = row_index(rows, r);
        const double* xi = x + (size_t)i * d;
        double acc[16];
        for (int c = 0; c < d; ++c) acc[c] = 0.0;
        for (int j = 0; j < T; ++j) {
            const double* xj = x + (size_t)j * d;
            double kij = exp(-sqdist(xj, xi, d) / (2.0 * h2));
            for (int c = 0; c < d; ++c)
                acc[c] += kij * score[(size_t)j * d + c] + kij * (xi[c] - xj[c]) / h2;
        }
        for (int c = 0; c < d; ++c) out[(size_t)r * d + c] = acc[c] / T;
    }
}

/* ------------------------------------------------------------------------
 * Reverse mode of the Stein field (Eq. 4) for a scalar L = <abar, g>:
 *   L = 1/T sum_i sum_j k_ij [ abar_i . s_j + abar_i . (x_i - x_j) / h^2 ],
 *   k_ij = exp(-|x_i - x_j|^2 / (2 h^2)),
 *   dk_ij/dx_i = -k_ij (x_i - x_j) / h^2 = -dk_ij/dx_j.
 * Product rule term by term, with phi_ij = abar_i . s_j + abar_i . (x_i - x_j) / h^2:
 *   sbar_j  = 1/T sum_i k_ij abar_i
 *   xbar_i += 1/T sum_j [ -k_ij (x_i - x_j) phi_ij / h^2 + k_ij abar_i / h^2 ]   (x_i as the row)
 *   xbar_j += 1/T sum_i [  k_ij (x_i - x_j) phi_ij / h^2 - k_ij abar_i / h^2 ]   (x_j as the column)
 * The score s is an input here (its own dependence on x is the mixture
 * score's reverse mode below).  Two plain passes, one per role of the
 * point, so that each output row is written by one loop iteration.
 * ---------------------------------------------------------------------- */
void orc_svgd_field_vjp(const double* x, int T, int d, const double* score,
                        double h, const double* abar, double* xbar,
                        double* sbar) {
    const double h2 = h * h;
#pragma omp parallel for schedule(static)
    for (int l = 0; l < T; ++l) {
        const double* xl = x + (size_t)l * d;
        double xr[16], xc[16], sc[16];
        for (int c = 0; c < d; ++c) xr[c] = xc[c] = sc[c] = 0.0;
        /* point l as the row i = l (sum over j) */
        for (int j = 0; j < T; ++j) {
            const double* xj = x + (size_t)j * d;
            double kij = exp(-sqdist(xl, xj, d) / (2.0 * h2));
            double phi = 0.0;
            for (int c = 0; c < d; ++c)
                phi += abar[(size_t)l * d + c] * (score[(size_t)j * d + c] + (xl[c] - xj[c]) / h2);
            for (int c = 0; c < d; ++c)
                xr[c] += -kij * (xl[c] - xj[c]) * phi / h2 + kij * abar[(size_t)l * d + c] / h2;
        }
        /* point l as the column j = l (sum over i) */
        for (int i = 0; i < T; ++i) {
            const double* xi = x + (size_t)i * d;
            double kil = exp(-sqdist(xi, xl, d) / (2.0 * h2));
            double phi = 0.0;
            for (int c = 0; c < d; ++c)
                phi += abar[(size_t)i * d + c] * (score[(size_t)l * d + c] + (xi[c] - xl[c]) / h2);
            for (int c = 0; c < d; ++c) {
                xc[c] += kil * (xi[c] - xl[c]) * phi / h2 - kil * abar[(size_t)i * d + c] / h2;
                sc[c] += kil * abar[(size_t)i * d + c];
            }
        }
        for (int c = 0; c < d; ++c) {
            xbar[(size_t)l * d + c] = (xr[c] + xc[c]) / T;
            if (sbar) sbar[(size_t)l * d + c] = sc[c] / T;
        }
    }
}

/* Reverse mode of the mixture score for the cotangents sbar_i of
 * score(x_i), i = 1..T.  With the component log terms
 *   t_k = log w_k - (d/2) log(2 pi sigma_k^2) - |x - mu_k|^2 / (2 sigma_k^2),
 * r = softmax(t), u_k = (mu_k - x) / sigma_k^2 and S = sum_k r_k u_k, a
 * change dt_k moves S by sum_k r_k (dt_k - sum_m r_m dt_m) u_k and a change
 * du_k by r_k du_k, so with c = sbar_i and beta_k = r_k (c . u_k - c . S):
 *   dt_k/dx = u_k, du_k/dx = -I / sigma_k^2:
 *     xbar += sum_k [ beta_k u_k - r_k c / sigma_k^2 ]
 *   dt_k/dmu_k = -u_k, du_k/dmu_k = I / sigma_k^2:
 *     mubar_k += -beta_k u_k + r_k c / sigma_k^2
 *   dt_k/dsigma_k = -d / sigma_k + |x - mu_k|^2 / sigma_k^3, du_k/dsigma_k = -2 u_k / sigma_k:
 *     sigmabar_k += beta_k (-d / sigma_k + |x - mu_k|^2 / sigma_k^3) - 2 r_k (c . u_k) / sigma_k
 *   dt_k/dw_k = 1 / w_k (the normalisation of w cancels in the softmax):
 *     wbar_k += beta_k / w_k
 * (sum_k beta_k u_k = sum_k r_k (c . u_k) (u_k - S), the Hessian of log q
 * applied to c.)  xbar_add, wbar, mubar, sigmabar may each be NULL; the
 * mixture gradients are sums over the T points. */
void orc_gmm_score_vjp(const double* x, int T, int d, int K, const double* w,
                       const double* mu, const double* sigma,
                       const double* sbar, double* xbar_add, double* wbar,
                       double* mubar, double* sigmabar) {
    if (wbar) for (int k = 0; k < K; ++k) wbar[k] = 0.0;
    if (mubar) for (int k = 0; k < K * d; ++k) mubar[k] = 0.0;
    if (sigmabar) for (int k = 0; k < K; ++k) sigmabar[k] = 0.0;
    double* t = (double*)malloc(sizeof(double) * K);
    double* u = (double*)malloc(sizeof(double) * (size_t)K * d);
    for (int i = 0; i < T; ++i) {
        const double* xi = x + (size_t)i * d;
        const double* c = sbar + (size_t)i * d;
        gmm_log_terms(xi, d, K, w, mu, sigma, t);
        double L = lse(t, K);
        double S[16], cS = 0.0;
        for (int a = 0; a < d; ++a) S[a] = 0.0;
        for (int k = 0; k < K; ++k) {
            double s2 = sigma[k] * sigma[k];
            t[k] = exp(t[k] - L); /* r_k */
            for (int a = 0; a < d; ++a) {
                u[(size_t)k * d + a] = (mu[(size_t)k * d + a] - xi[a]) / s2;
                S[a] += t[k] * u[(size_t)k * d + a];
            }
        }
        for (int a = 0; a < d; ++a) cS += c[a] * S[a];
        for (int k = 0; k < K; ++k) {
            double s2 = sigma[k] * sigma[k];
            double cu = 0.0, dist2 = 0.0;
            for (int a = 0; a < d; ++a) cu += c[a] * u[(size_t)k * d + a];
            dist2 = sqdist(xi, mu + (size_t)k * d, d);
            double beta = t[k] * (cu - cS);
            for (int a = 0; a < d; ++a) {
                double uka = u[(size_t)k * d + a];
                if (xbar_add) xbar_add[(size_t)i * d + a] += beta * uka - t[k] * c[a] / s2;
                if (mubar) mubar[(size_t)k * d + a] += -beta * uka + t[k] * c[a] / s2;
            }
            if (sigmabar)
                sigmabar[k] += beta * (-d / sigma[k] + dist2 / (s2 * sigma[k])) - 2.0 * t[k] * cu / sigma[k];
            if (wbar) wbar[k] += beta / w[k];
        }
    }
    free(t);
    free(u);
}

/* ------------------------------------------------------------------------
 * Entropic OT between p_s = sum_i a_i delta_{x_i} (a_i = 1/T, Eq. 1) and
 * q = sum_j b_j delta_{y_j} (Eq. 5), solved by the log-domain Sinkhorn
 * algorithm the paper cites for Eq. 6.  Reading of the garbled marginal
 * constraints of Eq. 5: probability marginals a and b.
 *
 * Dual potentials f (on x), g (on y); the half-step updates are
 *   g_j = -eps LSE_i( log a_i + (f_i - c(x_i, y_j)) / eps )
 *   f_i = -eps LSE_j( log b_j + (g_j - c(x_i, y_j)) / eps )
 * and the debiasing self-term OT(p_s, p_s) of Eq. 6 has one symmetric
 * potential p, updated by the averaged (Jacobi) step
 *   p_i <- 1/2 ( p_i - eps LSE_k( log a_k + (p_k - c(x_i, x_k)) / eps ) ).
 * ---------------------------------------------------------------------- */
/* Reference weights: b_j / sum_k b_k (NULL: uniform 1/M).  Reading: the
 * balanced problem needs equal total mass, so given weights are normalised
 * to a probability vector. */
static double wsum(const double* b, int M) {
    double s = 0.0;
    if (!b) return 1.0;
    for (int j = 0; j < M; ++j) s += b[j];
    return s;
}
static double wt(const double* b, int M, int j, double bs) {
    return b ? b[j] / bs : 1.0 / M;
}

void orc_sinkhorn_g_update(const double* x, int T, const double* y, int M,
                           int d, double eps, const double* f,
                           const int* rows, int n_rows, double* g_out) {
    int nr = rows ? n_rows : M;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nr; ++r) {
        int j = row_index(rows, r);
        double* z = (double*)malloc(sizeof(double) * T);
        for (int i = 0; i < T; ++i)
            z[i] = log(1.0 / T) + (f[i] - sqdist(x + (size_t)i * d, y + (size_t)j * d, d)) / eps;
        g_out[r] = -eps * lse(z, T);
        free(z);
    }
}

void orc_sinkhorn_f_update(const double* x, int T, const double* y, int M,
                           const double* b, int d, double eps,
                           const double* g, const int* rows, int n_rows,
                           double* f_out) {
    int nr = rows ? n_rows : T;
    double bs = wsum(b, M);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nr; ++r) {
        int i = row_index(rows, r);
        double* z = (double*)malloc(sizeof(double) * M);
        for (int j = 0; j < M; ++j)
            z[j] = log(wt(b, M, j, bs)) + (g[j] - sqdist(x + (size_t)i * d, y + (size_t)j * d, d)) / eps;
        f_out[r] = -eps * lse(z, M);
        free(z);
    }
}

/* Self-term update on a weighted point set (pts, w); w == NULL: uniform. */
static void self_update(const double* pts, int n, const double* w, int d,
                        double eps, const double* p_old, const int* rows,
                        int n_rows, double* p_out) {
    int nr = rows ? n_rows : n;
    double ws = wsum(w, n);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nr; ++r) {
        int i = row_index(rows, r);
        double* z = (double*)malloc(sizeof(double) * n);
        for (int k = 0; k < n; ++k)
            z[k] = log(wt(w, n, k, ws)) + (p_old[k] - sqdist(pts + (size_t)i * d, pts + (size_t)k * d, d)) / eps;
        p_out[r] = 0.5 * (p_old[i] - eps * lse(z, n));
        free(z);
    }
}

void orc_sinkhorn_p_update(const double* x, int T, int d, double eps,
                           const double* p_old, const int* rows, int n_rows,
                           double* p_out) {
    self_update(x, T, NULL, d, eps, p_old, rows, n_rows, p_out);
}

/* Fixed-iteration Sinkhorn.  Reading (the paper gives no schedule): cold
 * start f = g = p = 0 unless warm != 0; each iteration updates g, then f,
 * then p (p from the previous iteration on the right-hand side). */
void orc_sinkhorn(const double* x, int T, const double* y, int M,
                  const double* b, int d, double eps, int n_iter, int warm,
                  double* f, double* g, double* p) {
    if (!warm) {
        for (int i = 0; i < T; ++i) f[i] = 0.0, p[i] = 0.0;
        for (int j = 0; j < M; ++j) g[j] = 0.0;
    }
    double* pn = (double*)malloc(sizeof(double) * T);
    for (int it = 0; it < n_iter; ++it) {
        orc_sinkhorn_g_update(x, T, y, M, d, eps, f, NULL, 0, g);
        orc_sinkhorn_f_update(x, T, y, M, b, d, eps, g, NULL, 0, f);
        orc_sinkhorn_p_update(x, T, d, eps, p, NULL, 0, pn);
        memcpy(p, pn, sizeof(double) * T);
    }
    free(pn);
}

/* ------------------------------------------------------------------------
 * Reference given as a density on a pixel grid (Sec. II-A: q may be a
 * continuous function; the Stein field needs only its score).  Reading: q is
 * the bilinear interpolant of the pixel values map[iy][ix] (iy the row /
 * second coordinate), pixel centres at ((ix + 1/2)/W, (iy + 1/2)/H) on
 * [0,1]^2, each coordinate clamped to the outermost centres (constant
 * extension: no pull from outside the map).  score = grad q / q.
 * ---------------------------------------------------------------------- */
static void density_cell(int n, double xc, int* i0, double* f, int* inside) {
    double u = xc * n - 0.5;
    *inside = (u > 0.0 && u < n - 1.0);
    if (u < 0.0) u = 0.0;
    if (u > n - 1.0) u = n - 1.0;
    int i = (int)floor(u);
    if (i > n - 2) i = n - 2;
    *i0 = i;
    *f = u - i;
}

double orc_density_value(const double* map, int H, int W, const double* x) {
    int ix, iy, inx, iny;
    double fx, fy;
    density_cell(W, x[0], &ix, &fx, &inx);
    density_cell(H, x[1], &iy, &fy, &iny);
    const double q00 = map[(size_t)iy * W + ix], q10 = map[(size_t)iy * W + ix + 1];
    const double q01 = map[(size_t)(iy + 1) * W + ix], q11 = map[(size_t)(iy + 1) * W + ix + 1];
    return (1 - fx) * (1 - fy) * q00 + fx * (1 - fy) * q10 + (1 - fx) * fy * q01 + fx * fy * q11;
}

void orc_density_score(const double* map, int H, int W, const double* x, int T, double* score) {
    for (int i = 0; i < T; ++i) {
        const double* xi = x + (size_t)i * 2;
        int ix, iy, inx, iny;
        double fx, fy;
        density_cell(W, xi[0], &ix, &fx, &inx);
        density_cell(H, xi[1], &iy, &fy, &iny);
        const double q00 = map[(size_t)iy * W + ix], q10 = map[(size_t)iy * W + ix + 1];
        const double q01 = map[(size_t)(iy + 1) * W + ix], q11 = map[(size_t)(iy + 1) * W + ix + 1];
        const double q = (1 - fx) * (1 - fy) * q00 + fx * (1 - fy) * q10 + (1 - fx) * fy * q01 + fx * fy * q11;
        const double gx = inx ? W * ((1 - fy) * (q10 - q00) + fy * (q11 - q01)) : 0.0;
        const double gy = iny ? H * ((1 - fx) * (q01 - q00) + fx * (q11 - q10)) : 0.0;
        score[(size_t)i * 2] = gx / q;
        score[(size_t)i * 2 + 1] = gy / q;
    }
}

/* eps-scaling (annealing; not in the paper, a standard way to speed up
 * Sinkhorn at small eps): iteration t (0-based) runs the same g, f, p
 * updates at eps_t = max(eps, eps_start * eps_decay^t); the potentials are
 * carried over in their natural (cost) units.  eps_start <= eps gives
 * orc_sinkhorn exactly. */
double orc_anneal_eps(double eps, double eps_start, double eps_decay, int t) {
    double e = eps_start;
    for (int k = 0; k < t; ++k) e *= eps_decay;
    return e > eps ? e : eps;
}

void orc_sinkhorn_annealed(const double* x, int T, const double* y, int M,
                           const double* b, int d, double eps, int n_iter,
                           double eps_start, double eps_decay, int warm,
                           double* f, double* g, double* p) {
    if (!warm) {
        for (int i = 0; i < T; ++i) f[i] = 0.0, p[i] = 0.0;
        for (int j = 0; j < M; ++j) g[j] = 0.0;
    }
    double* pn = (double*)malloc(sizeof(double) * T);
    for (int it = 0; it < n_iter; ++it) {
        const double e = orc_anneal_eps(eps, eps_start, eps_decay, it);
        orc_sinkhorn_g_update(x, T, y, M, d, e, f, NULL, 0, g);
        orc_sinkhorn_f_update(x, T, y, M, b, d, e, g, NULL, 0, f);
        orc_sinkhorn_p_update(x, T, d, e, p, NULL, 0, pn);
        memcpy(p, pn, sizeof(double) * T);
    }
    free(pn);
}

/* ------------------------------------------------------------------------
 * Sinkhorn-divergence field, Eq. 7.  With the potentials held fixed
 * (envelope theorem), for c = |x - y|^2:
 *   grad_{x_i} OT(p_s, q)       = a_i sum_j pi_ij 2 (x_i - y_j)
 *   grad_{x_i} 1/2 OT(p_s, p_s) = a_i sum_k pi^s_ik 2 (x_i - x_k)
 *   grad_{x_i} OT(q, q)         = 0
 * with pi_ij = softmax_j(log b_j + (g_j - c_ij)/eps) and
 *      pi^s_ik = softmax_k(log a_k + (p_k - c_ik)/eps).
 * Reading of the sign/scale: the flow is the descent direction divided by
 * the sample weight a_i, i.e.  field_i = 2 (ybar_i - xbar_i).
 * ---------------------------------------------------------------------- */
static void bary(const double* xi, const double* pts, int n, const double* w,
                 const double* pot, int d, double eps, double* z,
                 double* out) {
    double ws = wsum(w, n);
    for (int k = 0; k < n; ++k)
        z[k] = log(wt(w, n, k, ws)) + (pot[k] - sqdist(xi, pts + (size_t)k * d, d)) / eps;
    double L = lse(z, n);
    for (int c = 0; c < d; ++c) out[c] = 0.0;
    for (int k = 0; k < n; ++k) {
        double pik = exp(z[k] - L);
        for (int c = 0; c < d; ++c) out[c] += pik * pts[(size_t)k * d + c];
    }
}

void orc_sinkhorn_field(const double* x, int T, const double* y, int M,
                        const double* b, int d, double eps, const double* g,
                        const double* p, const int* rows, int n_rows,
                        double* out) {
    int nr = rows ? n_rows : T;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nr; ++r) {
        int i = row_index(rows, r);
        const double* xi = x + (size_t)i * d;
        double* z = (double*)malloc(sizeof(double) * (M > T ? M : T));
        double yb[16], xb[16];
        bary(xi, y, M, b, g, d, eps, z, yb);
        bary(xi, x, T, NULL, p, d, eps, z, xb);
        for (int c = 0; c < d; ++c) out[(size_t)r * d + c] = 2.0 * (yb[c] - xb[c]);
        free(z);
    }
}

/* Marginals of pi_ij = a_i b_j exp((f_i + g_j - c_ij)/eps). */
void orc_sinkhorn_marginals(const double* x, int T, const double* y, int M,
                            const double* b, int d, double eps,
                            const double* f, const double* g,
                            double* row_sum, double* col_sum) {
    double bs = wsum(b, M);
    for (int i = 0; i < T; ++i) row_sum[i] = 0.0;
    for (int j = 0; j < M; ++j) col_sum[j] = 0.0;
    for (int i = 0; i < T; ++i)
        for (int j = 0; j < M; ++j) {
            double pij = (1.0 / T) * wt(b, M, j, bs) *
                         exp((f[i] + g[j] - sqdist(x + (size_t)i * d, y + (size_t)j * d, d)) / eps);
            row_sum[i] += pij;
            col_sum[j] += pij;
        }
}

/* Self-plan marginal error sum_i | sum_k w_i w_k exp((p_i+p_k-c_ik)/eps) - w_i |. */
static double self_marginal_err(const double* pts, int n, const double* w,
                                int d, double eps, const double* p) {
    double err = 0.0, ws = wsum(w, n);
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = 0; k < n; ++k)
            s += wt(w, n, i, ws) * wt(w, n, k, ws) *
                 exp((p[i] + p[k] - sqdist(pts + (size_t)i * d, pts + (size_t)k * d, d)) / eps);
        err += fabs(s - wt(w, n, i, ws));
    }
    return err;
}

static int self_converge(const double* pts, int n, const double* w, int d,
                         double eps, double tol, int max_iter, double* p) {
    double* pn = (double*)malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) p[i] = 0.0;
    int it;
    for (it = 1; it <= max_iter; ++it) {
        self_update(pts, n, w, d, eps, p, NULL, 0, pn);
        memcpy(p, pn, sizeof(double) * n);
        if (self_marginal_err(pts, n, w, d, eps, p) < tol) break;
    }
    free(pn);
    return it <= max_iter ? it : -max_iter;
}

/* Sinkhorn iterations until the column marginal (the row marginal is exact
 * after the f half-step) and the self-plan marginal are within tol (L1). */
int orc_sinkhorn_converge(const double* x, int T, const double* y, int M,
                          const double* b, int d, double eps, double tol,
                          int max_iter, double* f, double* g, double* p) {
    double* rs = (double*)malloc(sizeof(double) * T);
    double* cs = (double*)malloc(sizeof(double) * M);
    for (int i = 0; i < T; ++i) f[i] = 0.0;
    for (int j = 0; j < M; ++j) g[j] = 0.0;
    int it, done = 0;
    double bs = wsum(b, M);
    for (it = 1; it <= max_iter; ++it) {
        orc_sinkhorn_g_update(x, T, y, M, d, eps, f, NULL, 0, g);
        orc_sinkhorn_f_update(x, T, y, M, b, d, eps, g, NULL, 0, f);
        orc_sinkhorn_marginals(x, T, y, M, b, d, eps, f, g, rs, cs);
        double err = 0.0;
        for (int j = 0; j < M; ++j) err += fabs(cs[j] - wt(b, M, j, bs));
        if (err < tol) { done = 1; break; }
    }
    free(rs);
    free(cs);
    int its = self_converge(x, T, NULL, d, eps, tol, max_iter, p);
    if (!done || its < 0) return -max_iter;
    return it > its ? it : its;
}

/* Sinkhorn divergence of Eq. 6 at converged potentials.  The dual value of
 * OT(alpha, beta) is <a, f> + <b, g> (after an f half-step the entropic
 * correction term is exactly zero), and OT(alpha, alpha) = 2 <a, p>. */
double orc_sinkhorn_divergence(const double* x, int T, const double* y,
                               int M, const double* b, int d, double eps,
                               double tol, int max_iter) {
    double* f = (double*)malloc(sizeof(double) * T);
    double* g = (double*)malloc(sizeof(double) * M);
    double* p = (double*)malloc(sizeof(double) * T);
    double* q = (double*)malloc(sizeof(double) * M);
    orc_sinkhorn_converge(x, T, y, M, b, d, eps, tol, max_iter, f, g, p);
    self_converge(y, M, b, d, eps, tol, max_iter, q);
    double ot_xy = 0.0, ot_xx = 0.0, ot_yy = 0.0, bs = wsum(b, M);
    for (int i = 0; i < T; ++i) ot_xy += f[i] / T, ot_xx += 2.0 * p[i] / T;
    for (int j = 0; j < M; ++j)
        ot_xy += wt(b, M, j, bs) * g[j], ot_yy += 2.0 * wt(b, M, j, bs) * q[j];
    free(f);
    free(g);
    free(p);
    free(q);
    return ot_xy - 0.5 * ot_xx - 0.5 * ot_yy;
}

/* ------------------------------------------------------------------------
 * Dynamics.  The paper's dynamics are continuous (s' = f(s, u), Sec. II-A);
 * reading: explicit Euler s_{t+1} = s_t + dt f(s_t, u_t).
 *   single integrator  s = (p0, p1),          u = (u0, u1)
 *   double integrator  s = (p0, p1, v0, v1),  u = (acc0, acc1)
 *   unicycle           s = (x, y, theta),     u = (speed, turn rate)
 * ---------------------------------------------------------------------- */
int orc_model_dims(int model, int* n, int* m) {
    switch (model) {
        case ORC_SINGLE_INT: *n = 2; *m = 2; return 0;
        case ORC_DOUBLE_INT: *n = 4; *m = 2; return 0;
        case ORC_UNICYCLE: *n = 3; *m = 2; return 0;
    }
    return -1;
}

static void dynamics(int model, const double* s, const double* u, double* f) {
    switch (model) {
        case ORC_SINGLE_INT:
            f[0] = u[0];
            f[1] = u[1];
            break;
        case ORC_DOUBLE_INT:
            f[0] = s[2];
            f[1] = s[3];
            f[2] = u[0];
            f[3] = u[1];
            break;
        case ORC_UNICYCLE:
            f[0] = u[0] * cos(s[2]);
            f[1] = u[0] * sin(s[2]);
            f[2] = u[1];
            break;
    }
}

void orc_step(int model, const double* s, const double* u, double dt,
              double* s_next) {
    int n, m;
    orc_model_dims(model, &n, &m);
    double f[8];
    dynamics(model, s, u, f);
    for (int r = 0; r < n; ++r) s_next[r] = s[r] + dt * f[r];
}

void orc_rollout(int model, const double* s0, const double* u, int T,
                 double dt, double* s) {
    int n, m;
    orc_model_dims(model, &n, &m);
    for (int r = 0; r < n; ++r) s[r] = s0[r];
    for (int t = 0; t < T; ++t)
        orc_step(model, s + (size_t)t * n, u + (size_t)t * m, dt, s + (size_t)(t + 1) * n);
}

/* Eq. 8 for the Euler map: A_t = I + dt df/ds, B_t = dt df/du at (s_t, u_t). */
void orc_linearize(int model, const double* s, const double* u, int T,
                   double dt, double* A, double* B) {
    int n, m;
    orc_model_dims(model, &n, &m);
    for (int t = 0; t < T; ++t) {
        double* At = A + (size_t)t * n * n;
        double* Bt = B + (size_t)t * n * m;
        const double* st = s + (size_t)t * n;
        const double* ut = u + (size_t)t * m;
        for (int r = 0; r < n * n; ++r) At[r] = 0.0;
        for (int r = 0; r < n * m; ++r) Bt[r] = 0.0;
        for (int r = 0; r < n; ++r) At[r * n + r] = 1.0;
        switch (model) {
            case ORC_SINGLE_INT:
                Bt[0 * m + 0] = dt;
                Bt[1 * m + 1] = dt;
                break;
            case ORC_DOUBLE_INT:
                At[0 * n + 2] = dt;
                At[1 * n + 3] = dt;
                Bt[2 * m + 0] = dt;
                Bt[3 * m + 1] = dt;
                break;
            case ORC_UNICYCLE:
                At[0 * n + 2] = -dt * ut[0] * sin(st[2]);
                At[1 * n + 2] = dt * ut[0] * cos(st[2]);
                Bt[0 * m + 0] = dt * cos(st[2]);
                Bt[1 * m + 0] = dt * sin(st[2]);
                Bt[2 * m + 1] = dt;
                break;
        }
    }
}

/* ------------------------------------------------------------------------
 * LQR flow matching, Eq. 9-10, discretised on the time grid (the common dt
 * weight of both integrals cancels):
 *   min_v  sum_{t=1..T} |z_t - abar_t|_Q^2 + sum_{t=0..T-1} |v_t|_R^2
 *   s.t.   z_{t+1} = A_t z_t + B_t v_t,  z_0 = 0.
 * Value function V_t(z) = z'P_t z + 2 p_t'z + const; backward Riccati:
 *   S = R + B'P'B,  G = B'P'A,  h = B'p',  K = S^-1 G,  k = S^-1 h,
 *   P = Q_t + A'P'A - G'K,  p = -Q_t abar_t + A'p' - K'h,
 * with Q_t = Q for t >= 1, Q_0 = 0, P_T = Q, p_T = -Q abar_T; then
 *   v_t = -K_t z_t - k_t,  z_{t+1} = A_t z_t + B_t v_t.
 * abar is indexed abar[(t-1)*n + r] for t = 1..T.
 * ---------------------------------------------------------------------- */

/* Solve S X = Y for X (S is m x m SPD, Y is m x c) by Cholesky. */
static void chol_solve(const double* S, int m, const double* Y, int c,
                       double* X) {
    double L[64];
    memset(L, 0, sizeof(L));
    for (int i = 0; i < m; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = S[i * m + j];
            for (int k = 0; k < j; ++k) s -= L[i * m + k] * L[j * m + k];
            L[i * m + j] = (i == j) ? sqrt(s) : s / L[j * m + j];
        }
    for (int col = 0; col < c; ++col) {
        double w[8];
        for (int i = 0; i < m; ++i) {
            double s = Y[i * c + col];
            for (int k = 0; k < i; ++k) s -= L[i * m + k] * w[k];
            w[i] = s / L[i * m + i];
        }
        for (int i = m - 1; i >= 0; --i) {
            double s = w[i];
            for (int k = i + 1; k < m; ++k) s -= L[k * m + i] * X[k * c + col];
            X[i * c + col] = s / L[i * m + i];
        }
    }
}

void orc_lqr_track(const double* A, const double* B, const double* Q,
                   const double* R, const double* abar, int T, int n, int m,
                   double* v, double* z, double* P1) {
    double* K = (double*)malloc(sizeof(double) * (size_t)T * m * n);
    double* k = (double*)malloc(sizeof(double) * (size_t)T * m);
    double P[64], p[8], Pn[64], pn[8];
    /* P_T = Q, p_T = -Q abar_T */
    for (int r = 0; r < n * n; ++r) P[r] = Q[r];
    for (int r = 0; r < n; ++r) {
        p[r] = 0.0;
        for (int c = 0; c < n; ++c) p[r] -= Q[r * n + c] * abar[(size_t)(T - 1) * n + c];
    }
    for (int t = T - 1; t >= 0; --t) {
        const double* At = A + (size_t)t * n * n;
        const double* Bt = B + (size_t)t * n * m;
        double PA[64], PB[64], S[64], G[64], h[8];
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c) {
                PA[r * n + c] = 0.0;
                for (int q = 0; q < n; ++q) PA[r * n + c] += P[r * n + q] * At[q * n + c];
            }
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < m; ++c) {
                PB[r * m + c] = 0.0;
                for (int q = 0; q < n; ++q) PB[r * m + c] += P[r * n + q] * Bt[q * m + c];
            }
        for (int r = 0; r < m; ++r) {
            for (int c = 0; c < m; ++c) {
                S[r * m + c] = R[r * m + c];
                for (int q = 0; q < n; ++q) S[r * m + c] += Bt[q * m + r] * PB[q * m + c];
            }
            for (int c = 0; c < n; ++c) {
                G[r * n + c] = 0.0;
                for (int q = 0; q < n; ++q) G[r * n + c] += Bt[q * m + r] * PA[q * n + c];
            }
            h[r] = 0.0;
            for (int q = 0; q < n; ++q) h[r] += Bt[q * m + r] * p[q];
        }
        double* Kt = K + (size_t)t * m * n;
        double* kt = k + (size_t)t * m;
        chol_solve(S, m, G, n, Kt);
        chol_solve(S, m, h, 1, kt);
        for (int r = 0; r < n; ++r) {
            for (int c = 0; c < n; ++c) {
                double s = (t >= 1) ? Q[r * n + c] : 0.0;
                for (int q = 0; q < n; ++q) s += At[q * n + r] * PA[q * n + c];
                for (int q = 0; q < m; ++q) s -= G[q * n + r] * Kt[q * n + c];
                Pn[r * n + c] = s;
            }
            double s = 0.0;
            if (t >= 1)
                for (int c = 0; c < n; ++c) s -= Q[r * n + c] * abar[(size_t)(t - 1) * n + c];
            for (int q = 0; q < n; ++q) s += At[q * n + r] * p[q];
            for (int q = 0; q < m; ++q) s -= Kt[q * n + r] * h[q];
            pn[r] = s;
        }
        memcpy(P, Pn, sizeof(double) * n * n);
        memcpy(p, pn, sizeof(double) * n);
        if (t == 1 && P1) memcpy(P1, P, sizeof(double) * n * n);
    }
    /* forward pass */
    double* zt = z;
    for (int r = 0; r < n; ++r) zt[r] = 0.0;
    for (int t = 0; t < T; ++t) {
        const double* At = A + (size_t)t * n * n;
        const double* Bt = B + (size_t)t * n * m;
        const double* Kt = K + (size_t)t * m * n;
        const double* kt = k + (size_t)t * m;
        const double* zc = z + (size_t)t * n;
        double* vt = v + (size_t)t * m;
        double* zn = z + (size_t)(t + 1) * n;
        for (int r = 0; r < m; ++r) {
            vt[r] = -kt[r];
            for (int c = 0; c < n; ++c) vt[r] -= Kt[r * n + c] * zc[c];
        }
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int c = 0; c < n; ++c) s += At[r * n + c] * zc[c];
            for (int c = 0; c < m; ++c) s += Bt[r * m + c] * vt[c];
            zn[r] = s;
        }
    }
    free(K);
    free(k);
}

/* ------------------------------------------------------------------------
 * Outer iteration (Sec. II-C, last paragraph): evaluate the reference flow
 * a_t = g(s_t) on all time steps at once (Sec. II-B, "Reference flow on
 * state trajectory"), lift it to the state space (zero on the state
 * components that are not coverage coordinates), linearise, solve the LQR
 * problem for v*, update u <- u + eta v*, and roll the dynamics out again
 * from the fixed s_0.  Reading: the samples are s_1..s_T (s_0 cannot move,
 * z_0 = 0), the coverage coordinates are the first d state components, the
 * Sinkhorn potentials start cold in every field evaluation.
 * ---------------------------------------------------------------------- */
int orc_solve_ex(int model, int T, double dt, const double* s0, int field,
                 int d, const double* y, const double* b, int M, int K,
                 const double* gw, const double* gmu, const double* gsigma,
                 double eps, int n_iter, double h, const double* Q,
                 const double* R, double eta, int n_outer, double* u,
                 double* s, int warm, double eps_start, double eps_decay,
                 const double* density, int dens_h, int dens_w);

int orc_solve(int model, int T, double dt, const double* s0, int field,
              int d, const double* y, const double* b, int M, int K,
              const double* gw, const double* gmu, const double* gsigma,
              double eps, int n_iter, double h, const double* Q,
              const double* R, double eta, int n_outer, double* u,
              double* s) {
    return orc_solve_ex(model, T, dt, s0, field, d, y, b, M, K, gw, gmu, gsigma, eps, n_iter, h, Q, R, eta,
                        n_outer, u, s, 0, 0.0, 1.0, NULL, 0, 0);
}

/* Variant: warm != 0 keeps the Sinkhorn potentials from one outer iteration
 * to the next (the first starts cold); eps_start > eps anneals eps within
 * each field evaluation (orc_sinkhorn_annealed); density (dens_h x dens_w,
 * d = 2) replaces the mixture as the Stein field's reference. */
int orc_solve_ex(int model, int T, double dt, const double* s0, int field,
                 int d, const double* y, const double* b, int M, int K,
                 const double* gw, const double* gmu, const double* gsigma,
                 double eps, int n_iter, double h, const double* Q,
                 const double* R, double eta, int n_outer, double* u,
                 double* s, int warm, double eps_start, double eps_decay,
                 const double* density, int dens_h, int dens_w) {
    int n, m;
    if (orc_model_dims(model, &n, &m) != 0 || d > n) return -1;
    double* x = (double*)malloc(sizeof(double) * (size_t)T * d);
    double* a = (double*)malloc(sizeof(double) * (size_t)T * d);
    double* sc = (double*)malloc(sizeof(double) * (size_t)T * d);
    double* abar = (double*)malloc(sizeof(double) * (size_t)T * n);
    double* A = (double*)malloc(sizeof(double) * (size_t)T * n * n);
    double* Bm = (double*)malloc(sizeof(double) * (size_t)T * n * m);
    double* v = (double*)malloc(sizeof(double) * (size_t)T * m);
    double* z = (double*)malloc(sizeof(double) * (size_t)(T + 1) * n);
    double* f = (double*)malloc(sizeof(double) * (size_t)T);
    double* p = (double*)malloc(sizeof(double) * (size_t)T);
    double* g = (double*)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
    orc_rollout(model, s0, u, T, dt, s);
    for (int it = 0; it < n_outer; ++it) {
        for (int i = 0; i < T; ++i)
            for (int c = 0; c < d; ++c) x[(size_t)i * d + c] = s[(size_t)(i + 1) * n + c];
        if (field == ORC_FIELD_SVGD) {
            if (density)
                orc_density_score(density, dens_h, dens_w, x, T, sc);
            else
                orc_gmm_score(x, T, d, K, gw, gmu, gsigma, sc);
            orc_svgd_field(x, T, d, sc, h, NULL, 0, a);
        } else {
            orc_sinkhorn_annealed(x, T, y, M, b, d, eps, n_iter, eps_start, eps_decay, warm && it > 0, f, g, p);
            orc_sinkhorn_field(x, T, y, M, b, d, eps, g, p, NULL, 0, a);
        }
        for (int i = 0; i < T; ++i)
            for (int r = 0; r < n; ++r) abar[(size_t)i * n + r] = (r < d) ? a[(size_t)i * d + r] : 0.0;
        orc_linearize(model, s, u, T, dt, A, Bm);
        orc_lqr_track(A, Bm, Q, R, abar, T, n, m, v, z, NULL);
        for (size_t r = 0; r < (size_t)T * m; ++r) u[r] += eta * v[r];
        orc_rollout(model, s0, u, T, dt, s);
    }
    free(x); free(a); free(sc); free(abar); free(A); free(Bm);
    free(v); free(z); free(f); free(p); free(g);
    return 0;
}

/* ------------------------------------------------------------------------
 * Adjoints.  Reverse mode of the definitions above, written out by hand:
 * for every softmax-type update the derivative of -eps LSE_k(z_k) is
 * -eps pi_k dz_k with pi = softmax(z), and dc(x, y)/dx = 2 (x - y).
 * ---------------------------------------------------------------------- */
static void softmax_inplace(double* z, int n) {
    double L = lse(z, n);
    for (int k = 0; k < n; ++k) z[k] = exp(z[k] - L);
}

void orc_sinkhorn_field_vjp(const double* x, int T, const double* y, int M,
                            const double* b, int d, double eps, int n_iter,
                            const double* abar, double* xbar, double* ybar,
                            double* bbar) {
    const int n = n_iter;
    const double bs = wsum(b, M);
    double* F = (double*)calloc((size_t)(n + 1) * T, sizeof(double));
    double* G = (double*)calloc((size_t)(n + 1) * M, sizeof(double));
    double* Pp = (double*)calloc((size_t)(n + 1) * T, sizeof(double));
    /* forward with the potentials of every iteration (cold start) */
    for (int t = 1; t <= n; ++t) {
        orc_sinkhorn_g_update(x, T, y, M, d, eps, F + (size_t)(t - 1) * T, NULL, 0, G + (size_t)t * M);
        orc_sinkhorn_f_update(x, T, y, M, b, d, eps, G + (size_t)t * M, NULL, 0, F + (size_t)t * T);
        orc_sinkhorn_p_update(x, T, d, eps, Pp + (size_t)(t - 1) * T, NULL, 0, Pp + (size_t)t * T);
    }
    double* gbar = (double*)calloc(M, sizeof(double));
    double* fbar = (double*)calloc(T, sizeof(double));
    double* pbar = (double*)calloc(T, sizeof(double));
    double* pprev = (double*)calloc(T, sizeof(double));
    double* lbbar = (double*)calloc(M, sizeof(double));
    double* z = (double*)malloc(sizeof(double) * (M > T ? M : T));
    const double* g = G + (size_t)n * M;
    const double* p = Pp + (size_t)n * T;

    /* field_i = 2 (sum_j pi_ij y_j - sum_k pi^s_ik x_k), objective <abar, field> */
    for (int i = 0; i < T; ++i) {
        const double* xi = x + (size_t)i * d;
        double A[16], yb[16], Ay = 0.0;
        for (int j = 0; j < M; ++j)
            z[j] = log(wt(b, M, j, bs)) + (g[j] - sqdist(xi, y + (size_t)j * d, d)) / eps;
        softmax_inplace(z, M);
        for (int c = 0; c < d; ++c) {
            A[c] = 2.0 * abar[(size_t)i * d + c];
            yb[c] = 0.0;
            for (int j = 0; j < M; ++j) yb[c] += z[j] * y[(size_t)j * d + c];
            Ay += A[c] * yb[c];
        }
        for (int j = 0; j < M; ++j) {
            const double* yj = y + (size_t)j * d;
            double Ayj = 0.0;
            for (int c = 0; c < d; ++c) {
                ybar[(size_t)j * d + c] += A[c] * z[j];
                Ayj += A[c] * yj[c];
            }
            const double sb = z[j] * (Ayj - Ay);
            gbar[j] += sb / eps;
            lbbar[j] += sb;
            const double cb = -sb / eps;
            for (int c = 0; c < d; ++c) {
                xbar[(size_t)i * d + c] += cb * 2.0 * (xi[c] - yj[c]);
                ybar[(size_t)j * d + c] += cb * 2.0 * (yj[c] - xi[c]);
            }
        }
    }
    for (int i = 0; i < T; ++i) {
        const double* xi = x + (size_t)i * d;
        double Bv[16], xb[16], Bx = 0.0;
        for (int k = 0; k < T; ++k)
            z[k] = log(1.0 / T) + (p[k] - sqdist(xi, x + (size_t)k * d, d)) / eps;
        softmax_inplace(z, T);
        for (int c = 0; c < d; ++c) {
            Bv[c] = -2.0 * abar[(size_t)i * d + c];
            xb[c] = 0.0;
            for (int k = 0; k < T; ++k) xb[c] += z[k] * x[(size_t)k * d + c];
            Bx += Bv[c] * xb[c];
        }
        for (int k = 0; k < T; ++k) {
            const double* xk = x + (size_t)k * d;
            double Bxk = 0.0;
            for (int c = 0; c < d; ++c) {
                xbar[(size_t)k * d + c] += Bv[c] * z[k];
                Bxk += Bv[c] * xk[c];
            }
            const double sb = z[k] * (Bxk - Bx);
            pbar[k] += sb / eps;
            const double cb = -sb / eps;
            for (int c = 0; c < d; ++c) {
                xbar[(size_t)i * d + c] += cb * 2.0 * (xi[c] - xk[c]);
                xbar[(size_t)k * d + c] += cb * 2.0 * (xk[c] - xi[c]);
            }
        }
    }
    /* back through the iterations, last first */
    for (int t = n; t >= 1; --t) {
        const double* pold = Pp + (size_t)(t - 1) * T;
        const double* gt = G + (size_t)t * M;
        const double* fold = F + (size_t)(t - 1) * T;
        /* p^t = (p^{t-1} - eps LSE_k(log a_k + (p^{t-1}_k - c_ik)/eps)) / 2 */
        for (int i = 0; i < T; ++i) pprev[i] = 0.5 * pbar[i];
        for (int i = 0; i < T; ++i) {
            const double* xi = x + (size_t)i * d;
            for (int k = 0; k < T; ++k)
                z[k] = log(1.0 / T) + (pold[k] - sqdist(xi, x + (size_t)k * d, d)) / eps;
            softmax_inplace(z, T);
            for (int k = 0; k < T; ++k) {
                const double w = 0.5 * pbar[i] * z[k];
                const double* xk = x + (size_t)k * d;
                pprev[k] -= w;
                for (int c = 0; c < d; ++c) {
                    xbar[(size_t)i * d + c] += w * 2.0 * (xi[c] - xk[c]);
                    xbar[(size_t)k * d + c] += w * 2.0 * (xk[c] - xi[c]);
                }
            }
        }
        memcpy(pbar, pprev, sizeof(double) * T);
        /* f^t = -eps LSE_j(log b_j + (g^t_j - c_ij)/eps) */
        for (int i = 0; i < T; ++i) {
            const double* xi = x + (size_t)i * d;
            for (int j = 0; j < M; ++j)
                z[j] = log(wt(b, M, j, bs)) + (gt[j] - sqdist(xi, y + (size_t)j * d, d)) / eps;
            softmax_inplace(z, M);
            for (int j = 0; j < M; ++j) {
                const double w = fbar[i] * z[j];
                const double* yj = y + (size_t)j * d;
                gbar[j] -= w;
                lbbar[j] -= eps * w;
                for (int c = 0; c < d; ++c) {
                    xbar[(size_t)i * d + c] += w * 2.0 * (xi[c] - yj[c]);
                    ybar[(size_t)j * d + c] += w * 2.0 * (yj[c] - xi[c]);
                }
            }
        }
        for (int i = 0; i < T; ++i) fbar[i] = 0.0;
        /* g^t = -eps LSE_i(log a_i + (f^{t-1}_i - c_ij)/eps) */
        for (int j = 0; j < M; ++j) {
            const double* yj = y + (size_t)j * d;
            for (int i = 0; i < T; ++i)
                z[i] = log(1.0 / T) + (fold[i] - sqdist(x + (size_t)i * d, yj, d)) / eps;
            softmax_inplace(z, T);
            for (int i = 0; i < T; ++i) {
                const double w = gbar[j] * z[i];
                const double* xi = x + (size_t)i * d;
                fbar[i] -= w;
                for (int c = 0; c < d; ++c) {
                    xbar[(size_t)i * d + c] += w * 2.0 * (xi[c] - yj[c]);
                    ybar[(size_t)j * d + c] += w * 2.0 * (yj[c] - xi[c]);
                }
            }
        }
        for (int j = 0; j < M; ++j) gbar[j] = 0.0;
    }
    /* log of the normalised weights -> raw weights */
    if (b && bbar) {
        double S = 0.0;
        for (int j = 0; j < M; ++j) S += lbbar[j];
        for (int j = 0; j < M; ++j) bbar[j] += lbbar[j] / b[j] - S / bs;
    }
    free(F); free(G); free(Pp); free(gbar); free(fbar); free(pbar); free(pprev); free(lbbar); free(z);
}

/* Adjoint of abar -> v.  v solves (G'QG + R) v = G'Q abar with z = G v, so
 * abar_bar = Q G w with (G'QG + R) w = vbar: w minimises
 * sum_t z'_t Q z'_t + w_t'R w_t - 2 vbar_t'w_t, z' = G w, an LQR problem
 * with a linear control cost r_t = -vbar_t and no state target:
 *   k_t = S^-1 (B'p' + r_t),  p_t = A'p' - K'(B'p' + r_t),  p_T = 0. */
void orc_lqr_vjp(const double* A, const double* B, const double* Q,
                 const double* R, const double* vbar, int T, int n, int m,
                 double* abar_bar) {
    double* K = (double*)malloc(sizeof(double) * (size_t)T * m * n);
    double* k = (double*)malloc(sizeof(double) * (size_t)T * m);
    double P[64], p[8], Pn[64], pn[8];
    for (int r = 0; r < n * n; ++r) P[r] = Q[r];
    for (int r = 0; r < n; ++r) p[r] = 0.0;
    for (int t = T - 1; t >= 0; --t) {
        const double* At = A + (size_t)t * n * n;
        const double* Bt = B + (size_t)t * n * m;
        double PA[64], PB[64], S[64], G[64], hh[8];
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c) {
                PA[r * n + c] = 0.0;
                for (int q = 0; q < n; ++q) PA[r * n + c] += P[r * n + q] * At[q * n + c];
            }
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < m; ++c) {
                PB[r * m + c] = 0.0;
                for (int q = 0; q < n; ++q) PB[r * m + c] += P[r * n + q] * Bt[q * m + c];
            }
        for (int r = 0; r < m; ++r) {
            for (int c = 0; c < m; ++c) {
                S[r * m + c] = R[r * m + c];
                for (int q = 0; q < n; ++q) S[r * m + c] += Bt[q * m + r] * PB[q * m + c];
            }
            for (int c = 0; c < n; ++c) {
                G[r * n + c] = 0.0;
                for (int q = 0; q < n; ++q) G[r * n + c] += Bt[q * m + r] * PA[q * n + c];
            }
            hh[r] = -vbar[(size_t)t * m + r];
            for (int q = 0; q < n; ++q) hh[r] += Bt[q * m + r] * p[q];
        }
        double* Kt = K + (size_t)t * m * n;
        double* kt = k + (size_t)t * m;
        chol_solve(S, m, G, n, Kt);
        chol_solve(S, m, hh, 1, kt);
        for (int r = 0; r < n; ++r) {
            for (int c = 0; c < n; ++c) {
                double s = (t >= 1) ? Q[r * n + c] : 0.0;
                for (int q = 0; q < n; ++q) s += At[q * n + r] * PA[q * n + c];
                for (int q = 0; q < m; ++q) s -= G[q * n + r] * Kt[q * n + c];
                Pn[r * n + c] = s;
            }
            double s = 0.0;
            for (int q = 0; q < n; ++q) s += At[q * n + r] * p[q];
            for (int q = 0; q < m; ++q) s -= Kt[q * n + r] * hh[q];
            pn[r] = s;
        }
        memcpy(P, Pn, sizeof(double) * n * n);
        memcpy(p, pn, sizeof(double) * n);
    }
    double zc[8], zn[8], w[8];
    for (int r = 0; r < n; ++r) zc[r] = 0.0;
    for (int t = 0; t < T; ++t) {
        const double* At = A + (size_t)t * n * n;
        const double* Bt = B + (size_t)t * n * m;
        const double* Kt = K + (size_t)t * m * n;
        const double* kt = k + (size_t)t * m;
        for (int r = 0; r < m; ++r) {
            w[r] = -kt[r];
            for (int c = 0; c < n; ++c) w[r] -= Kt[r * n + c] * zc[c];
        }
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int c = 0; c < n; ++c) s += At[r * n + c] * zc[c];
            for (int c = 0; c < m; ++c) s += Bt[r * m + c] * w[c];
            zn[r] = s;
        }
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int c = 0; c < n; ++c) s += Q[r * n + c] * zn[c];
            abar_bar[(size_t)t * n + r] = s;
        }
        memcpy(zc, zn, sizeof(double) * n);
    }
    free(K);
    free(k);
}

/* s_{t+1} = F(s_t, u_t): lambda_T = sbar_T, u_bar_t = B_t' lambda_{t+1},
 * lambda_t = sbar_t + A_t' lambda_{t+1}; d/ds0 = lambda_0. */
void orc_rollout_vjp(int model, const double* s, const double* u, int T,
                     double dt, const double* sbar, double* ubar,
                     double* s0bar) {
    int n, m;
    orc_model_dims(model, &n, &m);
    double* A = (double*)malloc(sizeof(double) * (size_t)T * n * n);
    double* B = (double*)malloc(sizeof(double) * (size_t)T * n * m);
    orc_linearize(model, s, u, T, dt, A, B);
    double lam[8], ln[8];
    for (int r = 0; r < n; ++r) lam[r] = sbar[(size_t)T * n + r];
    for (int t = T - 1; t >= 0; --t) {
        const double* At = A + (size_t)t * n * n;
        const double* Bt = B + (size_t)t * n * m;
        for (int c = 0; c < m; ++c) {
            double acc = 0.0;
            for (int r = 0; r < n; ++r) acc += Bt[r * m + c] * lam[r];
            ubar[(size_t)t * m + c] = acc;
        }
        for (int c = 0; c < n; ++c) {
            double acc = sbar[(size_t)t * n + c];
            for (int r = 0; r < n; ++r) acc += At[r * n + c] * lam[r];
            ln[c] = acc;
        }
        memcpy(lam, ln, sizeof(double) * n);
    }
    for (int r = 0; r < n; ++r) s0bar[r] += lam[r];
    free(A);
    free(B);
}

/* Reverse sweep of the outer iteration (Sec. II-C) for time-invariant
 * dynamics, given the trajectories of every outer iteration (the
 * checkpoints s_hist[k] = s^k, k = 0..K-1, each [T+1][n]) and the loss
 * gradient sbar_K with respect to the final trajectory s^K.  With A, B
 * independent of the trajectory, v^k depends on s^{k-1} only through the
 * field, so
 *   ubar^K = rollout_vjp(sbar_K),
 *   for k = K..1:  abar_bar = lqr_vjp(eta ubar^k);
 *                  (xbar, ybar, bbar) += field_vjp(x^{k-1}; abar_bar);
 *                  ubar^{k-1} = ubar^k + rollout_vjp(lift(xbar)).
 * Outputs are accumulated into ybar [M][d], bbar [M] (may be NULL), s0bar [n]
 * and written to u0bar [T][m] (may be NULL).  Returns 0, or -1 for a
 * trajectory-dependent linearisation. */
int orc_solve_backward(int model, int T, double dt, int d, const double* y,
                       const double* b, int M, double eps, int n_iter,
                       const double* Q, const double* R, double eta,
                       int n_outer, const double* s_hist, const double* sbar_K,
                       double* ybar, double* bbar, double* s0bar,
                       double* u0bar) {
    int n, m;
    if (orc_model_dims(model, &n, &m) != 0 || model == ORC_UNICYCLE || d > n) return -1;
    const size_t us = (size_t)T * m, ss = (size_t)(T + 1) * n;
    double* A = (double*)malloc(sizeof(double) * (size_t)T * n * n);
    double* Bm = (double*)malloc(sizeof(double) * (size_t)T * n * m);
    double* ubar = (double*)calloc(us, sizeof(double));
    double* ub2 = (double*)calloc(us, sizeof(double));
    double* v = (double*)calloc(us, sizeof(double));
    double* u0 = (double*)calloc(us, sizeof(double));
    double* sbar = (double*)calloc(ss, sizeof(double));
    double* x = (double*)malloc(sizeof(double) * (size_t)T * d);
    double* xbar = (double*)calloc((size_t)T * d, sizeof(double));
    double* fa = (double*)calloc((size_t)T * d, sizeof(double));
    double* abb = (double*)calloc((size_t)T * n, sizeof(double));
    /* A, B do not depend on (s, u) for these models: take them anywhere */
    orc_linearize(model, s_hist, u0, T, dt, A, Bm);
    orc_rollout_vjp(model, s_hist, u0, T, dt, sbar_K, ubar, s0bar);
    for (int k = n_outer; k >= 1; --k) {
        const double* Sp = s_hist + (size_t)(k - 1) * ss;
        for (size_t r = 0; r < us; ++r) v[r] = eta * ubar[r];
        orc_lqr_vjp(A, Bm, Q, R, v, T, n, m, abb);
        for (int i = 0; i < T; ++i)
            for (int c = 0; c < d; ++c) {
                fa[(size_t)i * d + c] = abb[(size_t)i * n + c];
                x[(size_t)i * d + c] = Sp[(size_t)(i + 1) * n + c];
                xbar[(size_t)i * d + c] = 0.0;
            }
        orc_sinkhorn_field_vjp(x, T, y, M, b, d, eps, n_iter, fa, xbar, ybar, bbar);
        for (size_t r = 0; r < ss; ++r) sbar[r] = 0.0;
        for (int i = 0; i < T; ++i)
            for (int c = 0; c < d; ++c) sbar[(size_t)(i + 1) * n + c] = xbar[(size_t)i * d + c];
        orc_rollout_vjp(model, Sp, u0, T, dt, sbar, ub2, s0bar);
        for (size_t r = 0; r < us; ++r) ubar[r] += ub2[r];
    }
    if (u0bar) memcpy(u0bar, ubar, sizeof(double) * us);
    free(A); free(Bm); free(ubar); free(ub2); free(v); free(u0); free(sbar);
    free(x); free(xbar); free(fa); free(abb);
    return 0;
}

/* Gradient of the coverage loss through n_outer outer iterations (Sec. II-C)
 * by reverse mode with the trajectory of every outer iteration kept (the
 * checkpoints), for time-invariant dynamics.  The loss is the Sinkhorn
 * divergence of the final positions to (y_loss, b_loss); its gradient with
 * respect to the final positions is -(1/T) times the field at converged
 * potentials (the envelope theorem, exact at convergence). */
/* Reverse sweep of a Stein-field solve (Eq. 4 with a mixture reference) on a
 * time-invariant model, the same steps as orc_solve_backward: at outer
 * iteration k the LQR adjoint of eta ubar gives the field's cotangent, the
 * Stein field's reverse mode at x^{k-1} (with the mixture score at x^{k-1})
 * gives the cotangent of the points (kernel and score paths) and of the
 * mixture, and the rollout adjoint carries the points' cotangent to u and
 * s_0.  The mixture gradients of every outer iteration are summed. */
int orc_solve_backward_svgd(int model, int T, double dt, int d, int K, const double* w,
                            const double* mu, const double* sigma, double h,
                            const double* Q, const double* R, double eta, int n_outer,
                            const double* s_hist, const double* sbar_K, double* wbar,
                            double* mubar, double* sigmabar, double* s0bar,
                            double* u0bar) {
    int n, m;
    if (orc_model_dims(model, &n, &m) != 0 || model == ORC_UNICYCLE || d > n) return -1;
    const size_t us = (size_t)T * m, ss = (size_t)(T + 1) * n;
    double* A = (double*)malloc(sizeof(double) * (size_t)T * n * n);
    double* Bm = (double*)malloc(sizeof(double) * (size_t)T * n * m);
    double* ubar = (double*)calloc(us, sizeof(double));
    double* ub2 = (double*)calloc(us, sizeof(double));
    double* v = (double*)calloc(us, sizeof(double));
    double* u0 = (double*)calloc(us, sizeof(double));
    double* sbar = (double*)calloc(ss, sizeof(double));
    double* x = (double*)malloc(sizeof(double) * (size_t)T * d);
    double* score = (double*)malloc(sizeof(double) * (size_t)T * d);
    double* xbar = (double*)calloc((size_t)T * d, sizeof(double));
    double* scb = (double*)calloc((size_t)T * d, sizeof(double));
    double* fa = (double*)calloc((size_t)T * d, sizeof(double));
    double* abb = (double*)calloc((size_t)T * n, sizeof(double));
    double* wk = (double*)malloc(sizeof(double) * K);
    double* mk = (double*)malloc(sizeof(double) * (size_t)K * d);
    double* sk = (double*)malloc(sizeof(double) * K);
    for (int k = 0; k < K; ++k) wbar[k] = sigmabar[k] = 0.0;
    for (int k = 0; k < K * d; ++k) mubar[k] = 0.0;
    /* A, B do not depend on (s, u) for these models: take them anywhere */
    orc_linearize(model, s_hist, u0, T, dt, A, Bm);
    orc_rollout_vjp(model, s_hist, u0, T, dt, sbar_K, ubar, s0bar);
    for (int k = n_outer; k >= 1; --k) {
        const double* Sp = s_hist + (size_t)(k - 1) * ss;
        for (size_t r = 0; r < us; ++r) v[r] = eta * ubar[r];
        orc_lqr_vjp(A, Bm, Q, R, v, T, n, m, abb);
        for (int i = 0; i < T; ++i)
            for (int c = 0; c < d; ++c) {
                fa[(size_t)i * d + c] = abb[(size_t)i * n + c];
                x[(size_t)i * d + c] = Sp[(size_t)(i + 1) * n + c];
            }
        orc_gmm_score(x, T, d, K, w, mu, sigma, score);
        orc_svgd_field_vjp(x, T, d, score, h, fa, xbar, scb);
        orc_gmm_score_vjp(x, T, d, K, w, mu, sigma, scb, xbar, wk, mk, sk);
        for (int c = 0; c < K; ++c) wbar[c] += wk[c], sigmabar[c] += sk[c];
        for (int c = 0; c < K * d; ++c) mubar[c] += mk[c];
        for (size_t r = 0; r < ss; ++r) sbar[r] = 0.0;
        for (int i = 0; i < T; ++i)
            for (int c = 0; c < d; ++c) sbar[(size_t)(i + 1) * n + c] = xbar[(size_t)i * d + c];
        orc_rollout_vjp(model, Sp, u0, T, dt, sbar, ub2, s0bar);
        for (size_t r = 0; r < us; ++r) ubar[r] += ub2[r];
    }
    if (u0bar) memcpy(u0bar, ubar, sizeof(double) * us);
    free(A); free(Bm); free(ubar); free(ub2); free(v); free(u0); free(sbar);
    free(x); free(score); free(xbar); free(scb); free(fa); free(abb); free(wk); free(mk); free(sk);
    return 0;
}

double orc_solve_sinkhorn_grad(int model, int T, double dt, const double* s0,
                               int d, const double* y, const double* b, int M,
                               double eps, int n_iter, const double* Q,
                               const double* R, double eta, int n_outer,
                               const double* u0, const double* y_loss,
                               const double* b_loss, int M_loss,
                               double eps_loss, double* ybar, double* bbar,
                               double* s0bar) {
    int n, m;
    if (orc_model_dims(model, &n, &m) != 0 || model == ORC_UNICYCLE || d > n) return NAN;
    const size_t us = (size_t)T * m, ss = (size_t)(T + 1) * n;
    double* S = (double*)malloc(sizeof(double) * (size_t)(n_outer + 1) * ss);
    double* u = (double*)malloc(sizeof(double) * us);
    double* x = (double*)malloc(sizeof(double) * (size_t)T * d);
    double* a = (double*)malloc(sizeof(double) * (size_t)T * d);
    double* f = (double*)malloc(sizeof(double) * (size_t)T);
    double* g = (double*)malloc(sizeof(double) * (size_t)M_loss);
    double* p = (double*)malloc(sizeof(double) * (size_t)T);
    double* sbar = (double*)calloc(ss, sizeof(double));
    memcpy(u, u0, sizeof(double) * us);
    orc_rollout(model, s0, u, T, dt, S);
    for (int k = 1; k <= n_outer; ++k) {
        memcpy(S + (size_t)k * ss, S + (size_t)(k - 1) * ss, sizeof(double) * ss);
        orc_solve(model, T, dt, s0, ORC_FIELD_SINKHORN, d, y, b, M, 0, NULL, NULL, NULL, eps, n_iter,
                  0.0, Q, R, eta, 1, u, S + (size_t)k * ss);
    }
    const double* SK = S + (size_t)n_outer * ss;
    for (int i = 0; i < T; ++i)
        for (int c = 0; c < d; ++c) x[(size_t)i * d + c] = SK[(size_t)(i + 1) * n + c];
    const double L = orc_sinkhorn_divergence(x, T, y_loss, M_loss, b_loss, d, eps_loss, 1e-12, 100000);
    orc_sinkhorn_converge(x, T, y_loss, M_loss, b_loss, d, eps_loss, 1e-12, 100000, f, g, p);
    orc_sinkhorn_field(x, T, y_loss, M_loss, b_loss, d, eps_loss, g, p, NULL, 0, a);
    for (int i = 0; i < T; ++i)
        for (int c = 0; c < d; ++c) sbar[(size_t)(i + 1) * n + c] = -a[(size_t)i * d + c] / T;
    orc_solve_backward(model, T, dt, d, y, b, M, eps, n_iter, Q, R, eta, n_outer, S, sbar, ybar, bbar,
                       s0bar, NULL);
    free(S); free(u); free(x); free(a); free(f); free(g); free(p); free(sbar);
    return L;
}
