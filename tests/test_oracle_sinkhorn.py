"""Pins of the oracle's log-domain Sinkhorn, Sinkhorn divergence (Eq. 5-6)
and Sinkhorn-divergence field (Eq. 7).

Independent references used here: the scaling-domain (matrix) form of the
same Sinkhorn iterations written with scipy's distance matrix, the exact
assignment optimum from scipy's linear_sum_assignment, the eps -> infinity
limit, a hand-worked single pair, symmetry (y = x) and finite differences.
"""
import json
import os

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment
from scipy.spatial.distance import cdist

from paper_2511_11514_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _scaling_sinkhorn(x, y, b, eps, n_iter):
    """Kernel-matrix Sinkhorn (Cuturi 2013 form) with the same schedule as
    the oracle's reading: g first, then f, then the averaged self update.
    u = exp(f/eps), v = exp(g/eps), w = exp(p/eps)."""
    T, M = len(x), len(y)
    a = np.full(T, 1.0 / T)
    b = b / b.sum()
    K = np.exp(-cdist(x, y, "sqeuclidean") / eps)
    Ks = np.exp(-cdist(x, x, "sqeuclidean") / eps)
    u, w = np.ones(T), np.ones(T)
    for _ in range(n_iter):
        v = 1.0 / (K.T @ (a * u))
        u = 1.0 / (K @ (b * v))
        w = np.sqrt(w / (Ks @ (a * w)))
    return eps * np.log(u), eps * np.log(v), eps * np.log(w)


def test_fixed_iterations_match_scaling_form(orc):
    x = wl.random_points(23, 2, seed=1)
    y = wl.random_points(31, 2, seed=2)
    b = wl.random_weights(31, seed=3)
    eps = 0.08
    for n_iter in (1, 2, 7):
        f, g, p = orc.sinkhorn(x, y, b, eps, n_iter)
        f2, g2, p2 = _scaling_sinkhorn(x, y, b, eps, n_iter)
        np.testing.assert_allclose(f, f2, rtol=0, atol=1e-12)
        np.testing.assert_allclose(g, g2, rtol=0, atol=1e-12)
        np.testing.assert_allclose(p, p2, rtol=0, atol=1e-12)


def test_converged_marginals(orc):
    """Marginals of pi = a b exp((f+g-c)/eps), rebuilt with scipy's cost."""
    x = wl.random_points(20, 2, seed=4)
    y = wl.random_points(30, 2, seed=5)
    b = wl.random_weights(30, seed=6)
    eps = 0.05
    f, g, p, it = orc.sinkhorn_converge(x, y, b, eps, tol=1e-12)
    assert it > 0
    a = np.full(20, 1 / 20)
    b = b / b.sum()
    pi = a[:, None] * b[None, :] * np.exp((f[:, None] + g[None, :] - cdist(x, y, "sqeuclidean")) / eps)
    assert np.abs(pi.sum(1) - a).sum() <= 1e-10
    assert np.abs(pi.sum(0) - b).sum() <= 1e-10
    ps = a[:, None] * a[None, :] * np.exp((p[:, None] + p[None, :] - cdist(x, x, "sqeuclidean")) / eps)
    assert np.abs(ps.sum(1) - a).sum() <= 1e-10
    rs, cs = orc.sinkhorn_marginals(x, y, b, eps, f, g)
    np.testing.assert_allclose(rs, pi.sum(1), rtol=1e-12)
    np.testing.assert_allclose(cs, pi.sum(0), rtol=1e-12)


def test_single_pair_hand_example(orc):
    ex = json.load(open(GOLDEN))["sinkhorn_single_pair"]
    x, y, eps = np.array(ex["x"]), np.array(ex["y"]), ex["eps"]
    assert orc.sinkhorn_divergence(x, y, None, eps) == pytest.approx(ex["divergence"], rel=1e-12)
    f, g, p = orc.sinkhorn(x, y, None, eps, 3)
    np.testing.assert_allclose(orc.sinkhorn_field(x, y, None, eps, g, p), ex["field"], rtol=1e-12)


def test_large_eps_limit(orc):
    """eps -> infinity: pi -> a (x) b, so OT(x,y) -> E|x-y|^2 and the
    debiased divergence -> |mean x - mean y|^2, and every field vector ->
    2 (mean y - mean x)."""
    x = wl.random_points(12, 2, seed=7)
    y = wl.random_points(15, 2, seed=8) + 0.3
    b = wl.random_weights(15, seed=9)
    eps = 1e5
    dmu = (b / b.sum()) @ y - x.mean(0)
    assert orc.sinkhorn_divergence(x, y, b, eps) == pytest.approx(float(dmu @ dmu), rel=1e-5)
    f, g, p = orc.sinkhorn(x, y, b, eps, 5)
    fld = orc.sinkhorn_field(x, y, b, eps, g, p)
    np.testing.assert_allclose(fld, np.tile(2 * dmu, (12, 1)), rtol=1e-4)


def test_small_eps_reaches_assignment_optimum(orc):
    """eps -> 0 with T = M and uniform weights: OT(x,y) -> the optimal
    assignment cost, with 0 <= OT_eps - OT_0 <= eps log n (KL form)."""
    n = 7
    x = wl.random_points(n, 2, seed=10)
    y = wl.random_points(n, 2, seed=11)
    C = cdist(x, y, "sqeuclidean")
    r, c = linear_sum_assignment(C)
    ot0 = C[r, c].mean()
    eps = 5e-3
    f, g, p, it = orc.sinkhorn_converge(x, y, None, eps, tol=1e-11)
    assert it > 0
    ot = f.mean() + g.mean()
    assert -1e-10 <= ot - ot0 <= eps * np.log(n) + 1e-10


def test_field_vanishes_when_reference_equals_trajectory(orc):
    """y = x with equal weights: cross and self problems coincide, so the
    debiased field is zero (this fails if the self term is dropped)."""
    x = wl.random_points(16, 2, seed=12)
    eps = 0.03
    f, g, p, it = orc.sinkhorn_converge(x, x, None, eps, tol=1e-13)
    fld = orc.sinkhorn_field(x, x, None, eps, g, p)
    assert np.abs(fld).max() < 1e-9
    # without the debiasing term the field would not vanish
    f2, g2, p2 = orc.sinkhorn(x, x, None, eps, 0)
    assert np.abs(orc.sinkhorn_field(x, x, None, eps, g, np.full(16, -1e3))).max() > 1e-3


def test_translation_equivariance(orc):
    x = wl.random_points(9, 2, seed=13)
    y = wl.random_points(11, 2, seed=14)
    eps = 0.04
    sh = np.array([0.25, -0.5])  # exact binary fractions keep costs identical
    f, g, p = orc.sinkhorn(x, y, None, eps, 6)
    f2, g2, p2 = orc.sinkhorn(x + sh, y + sh, None, eps, 6)
    np.testing.assert_allclose(f2, f, atol=1e-12)
    np.testing.assert_allclose(p2, p, atol=1e-12)
    np.testing.assert_allclose(orc.sinkhorn_field(x + sh, y + sh, None, eps, g2, p2),
                               orc.sinkhorn_field(x, y, None, eps, g, p), atol=1e-12)


def test_field_is_scaled_descent_direction_of_divergence(orc):
    """Envelope theorem at convergence: dD/dx_i = -(1/T) field_i, checked by
    central finite differences (step 1e-6) of the divergence value."""
    T, M = 6, 7
    x = wl.random_points(T, 2, seed=15)
    y = wl.random_points(M, 2, seed=16)
    b = wl.random_weights(M, seed=17)
    eps = 0.1
    f, g, p, it = orc.sinkhorn_converge(x, y, b, eps, tol=1e-14)
    fld = orc.sinkhorn_field(x, y, b, eps, g, p)
    hstep = 1e-6
    for i in range(T):
        for c in range(2):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += hstep
            xm[i, c] -= hstep
            fd = (orc.sinkhorn_divergence(xp, y, b, eps, tol=1e-14) -
                  orc.sinkhorn_divergence(xm, y, b, eps, tol=1e-14)) / (2 * hstep)
            assert fd == pytest.approx(-fld[i, c] / T, rel=1e-5, abs=1e-8)


def test_row_updates_match_full_updates(orc):
    x = wl.random_points(19, 2, seed=18)
    y = wl.random_points(27, 2, seed=19)
    b = wl.random_weights(27, seed=20)
    eps = 0.02
    f, g, p = orc.sinkhorn(x, y, b, eps, 3)
    rows_y = np.array([0, 26, 3])
    rows_x = np.array([18, 0, 4])
    g_full = orc.sinkhorn_g_update(x, y, eps, f)
    np.testing.assert_array_equal(orc.sinkhorn_g_update(x, y, eps, f, rows=rows_y), g_full[rows_y])
    f_full = orc.sinkhorn_f_update(x, y, b, eps, g_full)
    np.testing.assert_array_equal(orc.sinkhorn_f_update(x, y, b, eps, g_full, rows=rows_x), f_full[rows_x])
    p_full = orc.sinkhorn_p_update(x, eps, p)
    np.testing.assert_array_equal(orc.sinkhorn_p_update(x, eps, p, rows=rows_x), p_full[rows_x])
    fld = orc.sinkhorn_field(x, y, b, eps, g, p)
    np.testing.assert_array_equal(orc.sinkhorn_field(x, y, b, eps, g, p, rows=rows_x), fld[rows_x])
    # one more iteration from the state = the fixed-iteration run of 4
    f4, g4, p4 = orc.sinkhorn(x, y, b, eps, 4)
    np.testing.assert_array_equal(g_full, g4)
    np.testing.assert_array_equal(f_full, f4)
    np.testing.assert_array_equal(p_full, p4)


# -- eps-scaling and warm starts (variants beyond the paper's cold fixed-eps loop) --
def test_anneal_schedule_closed_form(orc):
    for t in range(12):
        assert orc.anneal_eps(0.002, 0.05, 0.6, t) == pytest.approx(max(0.002, 0.05 * 0.6 ** t), rel=1e-15)
    assert orc.anneal_eps(0.01, 0.005, 0.5, 0) == 0.01          # start below target: no scaling


def test_annealed_without_scaling_is_the_plain_iteration(orc):
    x = wl.random_points(23, 2, seed=61)
    y = wl.random_points(31, 2, seed=62)
    b = wl.random_weights(31, seed=63)
    for u, v in zip(orc.sinkhorn_annealed(x, y, b, 0.02, 7, 0.0, 0.5), orc.sinkhorn(x, y, b, 0.02, 7)):
        np.testing.assert_array_equal(u, v)


def test_annealed_iterations_use_the_scheduled_eps(orc):
    """Iteration t runs the plain g, f, p updates at eps_t (checked for the
    first three iterations by composing the single updates)."""
    x = wl.random_points(17, 2, seed=64)
    y = wl.random_points(19, 2, seed=65)
    b = wl.random_weights(19, seed=66)
    eps, e0, dec = 0.01, 0.08, 0.5
    f, g, p = np.zeros(17), np.zeros(19), np.zeros(17)
    for t in range(3):
        e = max(eps, e0 * dec ** t)
        g = orc.sinkhorn_g_update(x, y, e, f)
        f = orc.sinkhorn_f_update(x, y, b, e, g)
        p = orc.sinkhorn_p_update(x, e, p)
    fa, ga, pa = orc.sinkhorn_annealed(x, y, b, eps, 3, e0, dec)
    np.testing.assert_allclose(fa, f, atol=1e-13)
    np.testing.assert_allclose(ga, g, atol=1e-13)
    np.testing.assert_allclose(pa, p, atol=1e-13)


def test_annealed_reaches_the_target_fixed_point_faster(orc):
    """At small eps the annealed iteration ends at the target problem's fixed
    point (same field as the converged potentials) and, for the same
    iteration count, closer to it than the cold iteration."""
    x = wl.random_points(60, 2, seed=67, lo=0.2, hi=0.8)
    y = wl.random_points(90, 2, seed=68)
    eps = 0.003
    f_c, g_c, p_c, _ = orc.sinkhorn_converge(x, y, None, eps, tol=1e-13)
    a_conv = orc.sinkhorn_field(x, y, None, eps, g_c, p_c)

    def marg_err(f, g):
        rs, cs = orc.sinkhorn_marginals(x, y, None, eps, f, g)
        return np.abs(cs - 1.0 / 90).sum()

    fa, ga, pa = orc.sinkhorn_annealed(x, y, None, eps, 1000, 0.1, 0.8)
    np.testing.assert_allclose(orc.sinkhorn_field(x, y, None, eps, ga, pa), a_conv, atol=1e-7)
    n = 40
    f1, g1, _ = orc.sinkhorn(x, y, None, eps, n)
    f2, g2, _ = orc.sinkhorn_annealed(x, y, None, eps, n, 0.1, 0.8)
    assert marg_err(f2, g2) < 0.5 * marg_err(f1, g1)


def test_warm_solve_carries_the_potentials(orc):
    """Two outer iterations with warm potentials = the second field evaluated
    from the first one's potentials (manual composition)."""
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=48, M=64)
    w = inst.wl
    eps, n_iter = 0.02, 5
    u2, s2 = orc.solve(w.model, w.dt, inst.s0, inst.u0, wl.FIELD_SINKHORN, inst.Q, inst.R, w.eta, 2, y=inst.y,
                       eps=eps, n_iter=n_iter, warm=True)
    u1c, s1c = orc.solve(w.model, w.dt, inst.s0, inst.u0, wl.FIELD_SINKHORN, inst.Q, inst.R, w.eta, 1, y=inst.y,
                         eps=eps, n_iter=n_iter)
    u1w, s1w = orc.solve(w.model, w.dt, inst.s0, inst.u0, wl.FIELD_SINKHORN, inst.Q, inst.R, w.eta, 1, y=inst.y,
                         eps=eps, n_iter=n_iter, warm=True)
    np.testing.assert_array_equal(s1w, s1c)                   # the first outer iteration starts cold
    s0tr = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    f, g, p = orc.sinkhorn(s0tr[1:, :2], inst.y, None, eps, n_iter)
    f, g, p = orc.sinkhorn(s1c[1:, :2], inst.y, None, eps, n_iter, f=f, g=g, p=p)
    a = orc.sinkhorn_field(s1c[1:, :2], inst.y, None, eps, g, p)
    A, B = orc.linearize(w.model, s1c, u1c, w.dt)
    abar = np.zeros((48, 4))
    abar[:, :2] = a
    v, _, _ = orc.lqr_track(A, B, inst.Q, inst.R, abar)
    np.testing.assert_allclose(u2, u1c + w.eta * v, atol=1e-12)


def test_fixed_iteration_divergence_single_pair(orc):
    """T = M = 1 (Eq. 6 by hand): after any n >= 1 the cross potentials are
    f = 0, g = c(x, y) and both self potentials are 0, so the dual value is
    |x - y|^2 exactly."""
    x, y = np.array([[0.2, 0.7]]), np.array([[0.5, 0.3]])
    for n in (1, 2, 9):
        assert orc.sinkhorn_divergence_iter(x, y, 0.03, n) == pytest.approx(0.25, abs=1e-14)


def test_fixed_iteration_divergence_matches_scaling_form(orc):
    """The dual value <a, f> + <b, g> - <a, p> - <b, q> from the kernel-matrix
    (scaling-domain) iterations with the same schedule, q from the self
    iteration of y."""
    x = wl.random_points(19, 2, seed=71)
    y = wl.random_points(27, 2, seed=72)
    eps, n = 0.05, 7
    f, g, p = _scaling_sinkhorn(x, y, np.ones(len(y)), eps, n)
    q = _scaling_sinkhorn(y, y, np.ones(len(y)), eps, n)[2]
    ref = f.mean() + g.mean() - p.mean() - q.mean()
    assert orc.sinkhorn_divergence_iter(x, y, eps, n) == pytest.approx(ref, rel=1e-11, abs=1e-14)


def test_fixed_iteration_divergence_converges_to_the_divergence(orc):
    """Many iterations reach the converged divergence of Eq. 6; y = x gives
    zero (debiasing)."""
    x = wl.random_points(9, 2, seed=73)
    y = wl.random_points(11, 2, seed=74)
    eps = 0.1
    conv = orc.sinkhorn_divergence(x, y, None, eps, tol=1e-14)
    assert orc.sinkhorn_divergence_iter(x, y, eps, 3000) == pytest.approx(conv, rel=1e-9, abs=1e-12)
    assert abs(orc.sinkhorn_divergence_iter(x, x, eps, 3000)) <= 1e-10


def test_permutation_and_rotation_equivariance(orc):
    """Relabelling the trajectory points permutes f, p and the field;
    relabelling the reference samples permutes g and changes nothing else;
    rotating both point sets by the same orthogonal map (the squared
    distance is rotation invariant) leaves the potentials and rotates the
    field (would catch a transposed operand or a swapped index)."""
    x = wl.random_points(10, 2, seed=21)
    y = wl.random_points(13, 2, seed=22)
    eps, n = 0.03, 7
    f, g, p = orc.sinkhorn(x, y, None, eps, n)
    a = orc.sinkhorn_field(x, y, None, eps, g, p)
    rng = np.random.default_rng(3)
    px, py = rng.permutation(10), rng.permutation(13)
    f2, g2, p2 = orc.sinkhorn(x[px], y[py], None, eps, n)
    np.testing.assert_allclose(f2, f[px], atol=1e-12)
    np.testing.assert_allclose(g2, g[py], atol=1e-12)
    np.testing.assert_allclose(p2, p[px], atol=1e-12)
    np.testing.assert_allclose(orc.sinkhorn_field(x[px], y[py], None, eps, g2, p2), a[px], atol=1e-12)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    f3, g3, p3 = orc.sinkhorn(x @ R.T, y @ R.T, None, eps, n)
    np.testing.assert_allclose(f3, f, atol=1e-10)
    np.testing.assert_allclose(g3, g, atol=1e-10)
    np.testing.assert_allclose(p3, p, atol=1e-10)
    np.testing.assert_allclose(orc.sinkhorn_field(x @ R.T, y @ R.T, None, eps, g3, p3), a @ R.T, atol=1e-10)
