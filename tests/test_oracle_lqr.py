"""Pins of the oracle's dynamics, linearisation (Eq. 8), LQR flow matching
(Eq. 9-10) and outer iteration.

Independent references: a dense KKT solve of the same quadratic program
(numpy), scipy's discrete algebraic Riccati solver, finite differences of the
step map, a hand-worked single step, and exact tracking as R -> 0.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

from paper_2511_11514_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _dense_kkt(A, B, Q, R, abar):
    """Stack z = G v (z_0 = 0) and solve the normal equations of
    sum_t |z_t - abar_t|_Q^2 + sum_t |v_t|_R^2 directly."""
    T, n, m = B.shape
    G = np.zeros((T * n, T * m))
    for s in range(T):              # v_s enters z_{s+1}, propagated by A
        blk = B[s]
        for t in range(s + 1, T + 1):
            G[(t - 1) * n:t * n, s * m:(s + 1) * m] = blk
            if t < T:
                blk = A[t] @ blk
    Qb = np.kron(np.eye(T), Q)
    Rb = np.kron(np.eye(T), R)
    v = np.linalg.solve(G.T @ Qb @ G + Rb, G.T @ Qb @ abar.reshape(-1))
    z = np.concatenate([np.zeros(n), G @ v]).reshape(T + 1, n)
    return v.reshape(T, m), z


@pytest.mark.parametrize("T,n,m,stable", [(1, 2, 2, False), (7, 3, 2, False), (40, 4, 2, False),
                                          (25, 4, 3, False), (600, 4, 2, True)])
def test_lqr_matches_dense_kkt(orc, T, n, m, stable):
    """Also at a long horizon (T = 600, A_t = 0.97 x random orthogonal), where
    a Riccati recursion that lets P lose symmetry drifts away."""
    g = wl.rng(100 + T)
    if stable:
        A = np.stack([0.97 * np.linalg.qr(g.standard_normal((n, n)))[0] for _ in range(T)])
    else:
        A = np.eye(n) + 0.1 * g.standard_normal((T, n, n))
    B = 0.3 * g.standard_normal((T, n, m))
    L = g.standard_normal((n, n))
    Q = L @ L.T / n + 0.1 * np.eye(n)
    Q[-1, :] = Q[:, -1] = 0.0          # PSD, as in the coverage weight
    Q[-1, -1] = 0.0
    Rm = g.standard_normal((m, m))
    R = 0.05 * (Rm @ Rm.T + np.eye(m))
    abar = g.standard_normal((T, n))
    v, z, _ = orc.lqr_track(A, B, Q, R, abar)
    v2, z2 = _dense_kkt(A, B, Q, R, abar)
    np.testing.assert_allclose(v, v2, rtol=1e-9, atol=1e-10 * np.abs(v2).max())
    np.testing.assert_allclose(z, z2, rtol=1e-9, atol=1e-10 * np.abs(z2).max())


def test_lqr_single_step_hand_example(orc):
    ex = json.load(open(GOLDEN))["lqr_single_step"]
    A = np.ones((1, 1, 1))
    B = np.full((1, 1, 1), ex["dt"])
    v, z, _ = orc.lqr_track(A, B, np.array([[ex["Q"]]]), np.array([[ex["R"]]]), np.array([[ex["abar"]]]))
    assert v[0, 0] == pytest.approx(ex["v0"], rel=1e-14)
    assert z[1, 0] == pytest.approx(ex["z1"], rel=1e-14)


def test_single_integrator_tracks_exactly_as_R_vanishes(orc):
    T, dt = 50, 0.1
    s = np.zeros((T + 1, 2))
    A, B = orc.linearize(wl.SINGLE_INT, s, np.zeros((T, 2)), dt)
    abar = wl.rng(3).standard_normal((T, 2))
    v, z, _ = orc.lqr_track(A, B, np.eye(2), 1e-14 * np.eye(2), abar)
    np.testing.assert_allclose(z[1:], abar, rtol=0, atol=1e-10)


def test_riccati_reaches_dare_fixed_point(orc):
    """Long horizon, constant (A, B, Q, R): P_1 -> the DARE solution."""
    dt = 0.05
    A1 = np.eye(4)
    A1[0, 2] = A1[1, 3] = dt
    B1 = np.zeros((4, 2))
    B1[2, 0] = B1[3, 1] = dt
    Q = np.diag([1.0, 1.0, 0.1, 0.1])
    R = 0.01 * np.eye(2)
    T = 3000
    A = np.broadcast_to(A1, (T, 4, 4)).copy()
    B = np.broadcast_to(B1, (T, 4, 2)).copy()
    _, _, P1 = orc.lqr_track(A, B, Q, R, np.zeros((T, 4)))
    X = scipy.linalg.solve_discrete_are(A1, B1, Q, R)
    np.testing.assert_allclose(P1, X, rtol=1e-8)


@pytest.mark.parametrize("model", [wl.SINGLE_INT, wl.DOUBLE_INT, wl.UNICYCLE])
def test_linearisation_matches_finite_differences(orc, model):
    n, m = wl.MODEL_DIMS[model]
    g = wl.rng(40 + model)
    T, dt = 5, 0.07
    s = g.standard_normal((T + 1, n))
    u = g.standard_normal((T, m))
    A, B = orc.linearize(model, s, u, dt)
    h = 1e-6
    for t in range(T):
        for c in range(n):
            e = np.zeros(n)
            e[c] = h
            fd = (orc.step(model, s[t] + e, u[t], dt) - orc.step(model, s[t] - e, u[t], dt)) / (2 * h)
            np.testing.assert_allclose(A[t][:, c], fd, atol=1e-8)
        for c in range(m):
            e = np.zeros(m)
            e[c] = h
            fd = (orc.step(model, s[t], u[t] + e, dt) - orc.step(model, s[t], u[t] - e, dt)) / (2 * h)
            np.testing.assert_allclose(B[t][:, c], fd, atol=1e-8)


def test_unicycle_step_closed_form(orc):
    s = np.array([0.1, 0.2, np.pi / 3])
    u = np.array([2.0, 0.5])
    dt = 0.1
    np.testing.assert_allclose(orc.step(wl.UNICYCLE, s, u, dt),
                               [0.1 + 0.2 * 0.5, 0.2 + 0.2 * np.sqrt(3) / 2, np.pi / 3 + 0.05], rtol=1e-15)


def test_rollout_chains_steps(orc):
    g = wl.rng(7)
    u = g.standard_normal((9, 2))
    s = orc.rollout(wl.UNICYCLE, np.array([0.1, 0.1, 0.3]), u, 0.05)
    for t in range(9):
        np.testing.assert_array_equal(s[t + 1], orc.step(wl.UNICYCLE, s[t], u[t], 0.05))


def test_linear_model_update_moves_state_by_eta_z(orc):
    """For linear dynamics the rollout is affine in u, so after u += eta v
    the new trajectory is s + eta z exactly (up to rounding)."""
    T, dt, eta = 30, 0.05, 0.4
    s0, u = wl.double_int_init(T, dt)
    u = u + 0.1 * wl.rng(1).standard_normal(u.shape)
    s = orc.rollout(wl.DOUBLE_INT, s0, u, dt)
    A, B = orc.linearize(wl.DOUBLE_INT, s, u, dt)
    abar = wl.rng(2).standard_normal((T, 4))
    v, z, _ = orc.lqr_track(A, B, wl.coverage_Q(wl.DOUBLE_INT), 0.01 * np.eye(2), abar)
    s_new = orc.rollout(wl.DOUBLE_INT, s0, u + eta * v, dt)
    np.testing.assert_allclose(s_new, s + eta * z, atol=1e-12)


def test_solve_one_iteration_composition(orc):
    """Single integrator, Q = I, R -> 0: one outer iteration moves every
    sample by eta times the field evaluated on the old trajectory."""
    inst = wl.make_instance(wl.SVGD_SINGLE_T256, T=64)
    w = inst.wl
    s = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    x = s[1:, :2]
    fld = orc.svgd_field(x, orc.gmm_score(x, *inst.gmm), w.h)
    u1, s1 = orc.solve(w.model, w.dt, inst.s0, inst.u0, wl.FIELD_SVGD, np.eye(2), 1e-14 * np.eye(2),
                       w.eta, 1, gmm=inst.gmm, h=w.h)
    np.testing.assert_allclose(s1[1:] - s[1:], w.eta * fld, rtol=0, atol=1e-9 * w.eta * np.abs(fld).max())
    np.testing.assert_array_equal(s1[0], inst.s0)


def test_solve_decreases_sinkhorn_divergence(orc):
    """A small Sinkhorn coverage problem: the divergence to the reference
    falls over the outer iterations (the method's purpose, Eq. 2)."""
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=96, M=192)
    w = inst.wl
    s = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    D0 = orc.sinkhorn_divergence(s[1:, :2], inst.y, None, 0.01, tol=1e-9)
    u, s5 = orc.solve(w.model, w.dt, inst.s0, inst.u0, wl.FIELD_SINKHORN, inst.Q, inst.R, w.eta, 8,
                      y=inst.y, eps=w.eps * 4, n_iter=30)
    D5 = orc.sinkhorn_divergence(s5[1:, :2], inst.y, None, 0.01, tol=1e-9)
    assert D5 < 0.5 * D0
