/*
 * cov_oracle.h -- plain FP64 CPU oracle for coverage trajectory synthesis as
 * statistical inference (Sun, Kwon, Murphey, arXiv 2511.11514).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test-suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or helper with the CUDA library, and neither
 * side includes or links the other.
 *
 * Conventions (all FP64, all arrays row-major, caller-owned host memory):
 *   x  [T][d]   trajectory sample points (coverage coordinates of s_1..s_T)
 *   y  [M][d]   reference samples, weights b [M] (NULL = uniform 1/M;
 *               given weights are normalised to sum 1)
 *   a_i = 1/T   trajectory sample weights (Eq. 1, uniform time grid)
 *   c(x,y) = |x - y|^2   (Sec. II-B, "squared norm")
 *   eps         entropic weight (the paper's omega in Eq. 5)
 *   rows/n_rows optional row subset (rows == NULL: every row, n_rows ignored);
 *               output row r of the subset is written at out[r*...].
 */
#ifndef COV_ORACLE_H
#define COV_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Dynamics models (explicit Euler of the continuous models, Eq. 3 / Eq. 8). */
enum { ORC_SINGLE_INT = 0, ORC_DOUBLE_INT = 1, ORC_UNICYCLE = 2 };

void orc_set_threads(int n);
int orc_get_threads(void);

/* ---- reference distribution: isotropic Gaussian mixture ---------------- */
double orc_gmm_logpdf(const double* x, int d, int K, const double* w,
                      const double* mu, const double* sigma);
void orc_gmm_score(const double* x, int T, int d, int K, const double* w,
                   const double* mu, const double* sigma, double* score);

/* ---- Stein variational field, Eq. 4 ------------------------------------ */
void orc_svgd_field(const double* x, int T, int d, const double* score,
                    double h, const int* rows, int n_rows, double* out);
/* Reverse mode of Eq. 4 for L = <abar, field>: xbar [T][d] (the score held
 * fixed) and sbar [T][d] = dL/dscore (may be NULL). */
void orc_svgd_field_vjp(const double* x, int T, int d, const double* score,
                        double h, const double* abar, double* xbar,
                        double* sbar);
/* Reverse mode of the mixture score for cotangents sbar [T][d] of
 * score(x_i): adds J(x_i)' sbar_i to xbar_add [T][d]; writes the gradients
 * of sum_i sbar_i . score(x_i) with respect to w [K] (raw weights),
 * mu [K][d], sigma [K].  Any output may be NULL. */
void orc_gmm_score_vjp(const double* x, int T, int d, int K, const double* w,
                       const double* mu, const double* sigma,
                       const double* sbar, double* xbar_add, double* wbar,
                       double* mubar, double* sigmabar);

/* ---- log-domain Sinkhorn, Eq. 5-6 -------------------------------------- */
void orc_sinkhorn_g_update(const double* x, int T, const double* y, int M,
                           int d, double eps, const double* f,
                           const int* rows, int n_rows, double* g_out);
void orc_sinkhorn_f_update(const double* x, int T, const double* y, int M,
                           const double* b, int d, double eps,
                           const double* g, const int* rows, int n_rows,
                           double* f_out);
void orc_sinkhorn_p_update(const double* x, int T, int d, double eps,
                           const double* p_old, const int* rows, int n_rows,
                           double* p_out);
void orc_sinkhorn(const double* x, int T, const double* y, int M,
                  const double* b, int d, double eps, int n_iter,
                  int warm, double* f, double* g, double* p);
/* ---- Sinkhorn-divergence field, Eq. 7 (descent direction, 1/a_i scaled) */
void orc_sinkhorn_field(const double* x, int T, const double* y, int M,
                        const double* b, int d, double eps, const double* g,
                        const double* p, const int* rows, int n_rows,
                        double* out);
/* Converged potentials; returns iterations used (negative = not converged). */
int orc_sinkhorn_converge(const double* x, int T, const double* y, int M,
                          const double* b, int d, double eps, double tol,
                          int max_iter, double* f, double* g, double* p);
void orc_sinkhorn_marginals(const double* x, int T, const double* y, int M,
                            const double* b, int d, double eps,
                            const double* f, const double* g,
                            double* row_sum, double* col_sum);
double orc_sinkhorn_divergence(const double* x, int T, const double* y,
                               int M, const double* b, int d, double eps,
                               double tol, int max_iter);

/* ---- dynamics, linearisation (Eq. 8), rollout --------------------------- */
int orc_model_dims(int model, int* n, int* m);
void orc_step(int model, const double* s, const double* u, double dt,
              double* s_next);
void orc_linearize(int model, const double* s, const double* u, int T,
                   double dt, double* A, double* B);
void orc_rollout(int model, const double* s0, const double* u, int T,
                 double dt, double* s);

/* ---- LQR tracking, Eq. 9-10 (discrete Riccati) ------------------------- */
void orc_lqr_track(const double* A, const double* B, const double* Q,
                   const double* R, const double* abar, int T, int n, int m,
                   double* v, double* z, double* P1);

/* ---- outer iteration (Sec. II-C, last paragraph) ----------------------- */
enum { ORC_FIELD_SVGD = 0, ORC_FIELD_SINKHORN = 1 };
double orc_anneal_eps(double eps, double eps_start, double eps_decay, int t);
void orc_sinkhorn_annealed(const double* x, int T, const double* y, int M, const double* b, int d, double eps, int n_iter, double eps_start, double eps_decay, int warm, double* f, double* g, double* p);
int orc_solve_ex(int model, int T, double dt, const double* s0, int field, int d, const double* y, const double* b, int M, int K, const double* gw, const double* gmu, const double* gsigma, double eps, int n_iter, double h, const double* Q, const double* R, double eta, int n_outer, double* u, double* s, int warm, double eps_start, double eps_decay, const double* density, int dens_h, int dens_w);
double orc_density_value(const double* map, int H, int W, const double* x);
void orc_density_score(const double* map, int H, int W, const double* x, int T, double* score);
int orc_solve(int model, int T, double dt, const double* s0, int field,
              int d, const double* y, const double* b, int M, int K,
              const double* gw, const double* gmu, const double* gsigma,
              double eps, int n_iter, double h, const double* Q,
              const double* R, double eta, int n_outer, double* u,
              double* s);

/* ---- adjoints (reverse mode of the definitions above) ------------------- */
/* Vector-Jacobian product of the Sinkhorn-divergence field (orc_sinkhorn with
 * n_iter cold-start iterations followed by orc_sinkhorn_field) with respect
 * to x, y and the raw weights b (normalised inside): given abar [T][d],
 * xbar += d<abar, field>/dx, ybar += .../dy, bbar += .../db (bbar may be NULL;
 * ignored when b == NULL). */
void orc_sinkhorn_field_vjp(const double* x, int T, const double* y, int M,
                            const double* b, int d, double eps, int n_iter,
                            const double* abar, double* xbar, double* ybar,
                            double* bbar);
/* Adjoint of the linear map abar -> v of orc_lqr_track: given vbar [T][m],
 * returns abar_bar [T][n] (row t-1 for target t = 1..T). */
void orc_lqr_vjp(const double* A, const double* B, const double* Q,
                 const double* R, const double* vbar, int T, int n, int m,
                 double* abar_bar);
/* Adjoint of orc_rollout: given sbar [T+1][n], returns ubar [T][m] and adds
 * d/ds0 to s0bar [n] (A_t, B_t at the rollout's own (s_t, u_t)). */
void orc_rollout_vjp(int model, const double* s, const double* u, int T,
                     double dt, const double* sbar, double* ubar,
                     double* s0bar);
/* Gradient of the coverage loss L = converged Sinkhorn divergence (weight
 * eps_loss) between the positions of the final trajectory and (y_loss, b_loss)
 * after n_outer Sinkhorn-field outer iterations, with respect to the field's
 * reference samples y [M][d], raw weights b [M] (may be NULL) and s0 [n].
 * Time-invariant models only (single / double integrator).  Returns L. */
int orc_solve_backward(int model, int T, double dt, int d, const double* y, const double* b, int M, double eps, int n_iter, const double* Q, const double* R, double eta, int n_outer, const double* s_hist, const double* sbar_K, double* ybar, double* bbar, double* s0bar, double* u0bar);
/* Reverse sweep of a Stein-field solve with a mixture reference (time-
 * invariant model): the gradients of L(s^K) given dL/ds^K = sbar_K and the
 * checkpoints s_hist [n_outer][T+1][n], with respect to the mixture's raw
 * weights wbar [K], means mubar [K][d], standard deviations sigmabar [K]
 * (summed over the outer iterations), s0bar [n] (accumulated into) and
 * u0bar [T][m] (or NULL).  Returns 0, or -1 for an unsupported model. */
int orc_solve_backward_svgd(int model, int T, double dt, int d, int K, const double* w,
                            const double* mu, const double* sigma, double h,
                            const double* Q, const double* R, double eta, int n_outer,
                            const double* s_hist, const double* sbar_K, double* wbar,
                            double* mubar, double* sigmabar, double* s0bar,
                            double* u0bar);
double orc_solve_sinkhorn_grad(int model, int T, double dt, const double* s0,
                               int d, const double* y, const double* b, int M,
                               double eps, int n_iter, const double* Q,
                               const double* R, double eta, int n_outer,
                               const double* u0, const double* y_loss,
                               const double* b_loss, int M_loss,
                               double eps_loss, double* ybar, double* bbar,
                               double* s0bar);

#ifdef __cplusplus
}
#endif
#endif
