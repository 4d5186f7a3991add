"""GPU parity of the Stein field (Eq. 4), the mixture score, linearisation
(Eq. 8), rollout and the FP64 LQR step (Eq. 9-10) with the FP64 oracle."""
import dataclasses

import numpy as np
import pytest
import torch

from conftest import dev32, dev64, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("T,d,K", [(1, 2, 1), (2, 2, 3), (37, 1, 2), (256, 2, 3), (1000, 3, 4), (4099, 2, 16),
                                   (300, 6, 5), (31, 2, 2), (33, 3, 2), (1024, 2, 3), (1025, 2, 3), (896, 6, 3),
                                   (897, 6, 2)])
def test_svgd_field_with_mixture_score(cov, ctx, orc, T, d, K):
    """Both paths against the oracle: the one-launch kernel (T <= 1024, and
    for d = 6 T <= 896 by its shared memory; 32 rows per CTA, ragged last
    block) and the all-pairs kernel past them."""
    w, mu, sigma = wl.gmm_params(K, seed=T + K, d=d)
    w, mu, sigma = (wl.f32_pair(v)[1] for v in (w, mu, sigma))
    x = wl.random_points(T, d, seed=T)
    h = 0.05 if d <= 2 else 0.2
    a = cov.cov_field_svgd(ctx, dev32(x), h, gmm=(w, mu, sigma))
    ao = orc.svgd_field(x, orc.gmm_score(x, w, mu, sigma), h)
    assert rel_norm(host(a), ao) <= 1e-4
    assert ctx.device_status()[1] == 0


@pytest.mark.parametrize("T", [700, 4099])
def test_svgd_field_permutation_and_rotation_equivariance(cov, ctx, T):
    """Both Stein paths (one launch at T = 700, all pairs at T = 4099):
    relabelled points give the relabelled field, and rotating the points and
    the mixture's means together rotates it (within FP32 rounding)."""
    w, mu, sigma = (wl.f32_pair(v)[1] for v in wl.gmm_params(5, seed=T, d=2))
    x = wl.random_points(T, 2, seed=T + 1)
    gmm = (w, mu, sigma)
    a = host(cov.cov_field_svgd(ctx, dev32(x), 0.05, gmm=gmm))
    perm = np.random.default_rng(T).permutation(T)
    assert rel_norm(host(cov.cov_field_svgd(ctx, dev32(x[perm]), 0.05, gmm=gmm)), a[perm]) <= 1e-5
    R = np.array([[0.6, -0.8], [0.8, 0.6]])  # exact in binary to a few ulps
    a_r = host(cov.cov_field_svgd(ctx, dev32(x @ R.T), 0.05, gmm=(w, mu @ R.T, sigma)))
    assert rel_norm(a_r, a @ R.T) <= 1e-4
    assert ctx.device_status()[1] == 0


@pytest.mark.parametrize("T,d", [(5, 2), (777, 2), (2500, 3)])
def test_svgd_field_with_given_score(cov, ctx, orc, T, d):
    x = wl.random_points(T, d, seed=1)
    sc = wl.f32_pair(wl.rng(2).standard_normal((T, d)) * 10)[1]
    a = cov.cov_field_svgd(ctx, dev32(x), 0.1, score=dev32(sc))
    assert rel_norm(host(a), orc.svgd_field(x, sc, 0.1)) <= 1e-4


def test_gmm_score(cov, ctx, orc):
    w, mu, sigma = (wl.f32_pair(v)[1] for v in wl.gmm_params(7, seed=3))
    x = wl.random_points(3000, 2, seed=4)
    sc = cov.cov_gmm_score(ctx, dev32(x), (w, mu, sigma))
    assert rel_norm(host(sc), orc.gmm_score(x, w, mu, sigma)) <= 1e-5


def _random_lqr(T, n, m, seed):
    """Time-varying, well-conditioned: A_t = 0.97 x (random orthogonal)."""
    g = wl.rng(seed)
    A = np.stack([0.97 * np.linalg.qr(g.standard_normal((n, n)))[0] for _ in range(T)])
    B = 0.3 * g.standard_normal((T, n, m))
    L = g.standard_normal((n, n))
    Q = L @ L.T / n + 0.1 * np.eye(n)
    Rm = g.standard_normal((m, m))
    R = 0.05 * (Rm @ Rm.T + np.eye(m))
    abar = g.standard_normal((T, n))
    return A, B, Q, R, abar


@pytest.mark.parametrize("T,n,m", [(1, 2, 2), (2, 1, 1), (33, 4, 2), (63, 4, 2), (64, 4, 2), (100, 3, 2),
                                   (150, 4, 2), (300, 3, 3), (700, 2, 2), (1000, 4, 3), (2500, 3, 2), (4096, 4, 2),
                                   (7000, 4, 3), (65, 2, 1), (70, 3, 3), (20000, 4, 2), (65536, 3, 2)])
def test_lqr_track_matches_oracle(cov, ctx, orc, T, n, m):
    """Horizons across the parallel plans: the serial pass (T < 64), and
    the Riccati recursion and affine scans with 0 to 3 grouping levels above
    their chunks (the depth grows with T)."""
    A, B, Q, R, abar = _random_lqr(T, n, m, seed=T + 10 * n + m)
    v, z = cov.cov_lqr_track(ctx, dev64(A), dev64(B), Q, R, dev64(abar))
    vo, zo, _ = orc.lqr_track(A, B, Q, R, abar)
    np.testing.assert_allclose(host(v), vo, rtol=1e-9, atol=1e-10 * np.abs(vo).max())
    np.testing.assert_allclose(host(z), zo, rtol=1e-9, atol=1e-10 * np.abs(zo).max())
    assert ctx.device_status()[1] == 0


@pytest.mark.parametrize("T,n,m", [(3, 1, 1), (127, 2, 2), (128, 2, 1), (129, 2, 3), (255, 2, 2), (256, 3, 3),
                                   (511, 2, 2), (512, 2, 3), (513, 2, 2), (1023, 1, 2), (1024, 1, 3), (1025, 1, 1)])
def test_lqr_short_horizon_kernel(cov, ctx, orc, T, n, m):
    """The one-CTA kernel of both affine recursions (n = 1 up to T = 1024,
    n = 2 up to T = 512; 128 lanes, so one step per lane up to T = 128 and
    ragged last chunks past it), and the first horizons past its range,
    against the oracle."""
    A, B, Q, R, abar = _random_lqr(T, n, m, seed=3 * T + 10 * n + m)
    v, z = cov.cov_lqr_track(ctx, dev64(A), dev64(B), Q, R, dev64(abar))
    vo, zo, _ = orc.lqr_track(A, B, Q, R, abar)
    np.testing.assert_allclose(host(v), vo, rtol=1e-9, atol=1e-10 * np.abs(vo).max())
    np.testing.assert_allclose(host(z), zo, rtol=1e-9, atol=1e-10 * np.abs(zo).max())
    assert ctx.device_status()[1] == 0


def test_lqr_double_integrator_long_horizon(cov, ctx, orc):
    """The benchmark's LQR: double integrator, coverage weight on position
    only (Q PSD), R = 0.01 I, T = 4096."""
    T, dt = 4096, 0.05
    s = np.zeros((T + 1, 4))
    A, B = orc.linearize(wl.DOUBLE_INT, s, np.zeros((T, 2)), dt)
    abar = np.zeros((T, 4))
    abar[:, :2] = wl.rng(5).standard_normal((T, 2)) * 0.1
    Q, R = wl.coverage_Q(wl.DOUBLE_INT), 0.01 * np.eye(2)
    v, z = cov.cov_lqr_track(ctx, dev64(A), dev64(B), Q, R, dev64(abar))
    vo, zo, _ = orc.lqr_track(A, B, Q, R, abar)
    np.testing.assert_allclose(host(v), vo, rtol=1e-9, atol=1e-11 * np.abs(vo).max())
    np.testing.assert_allclose(host(z), zo, rtol=1e-9, atol=1e-11 * np.abs(zo).max())
    assert ctx.device_status()[1] == 0


@pytest.mark.parametrize("T", [8, 200])
def test_lqr_reports_non_spd_riccati(cov, ctx, T):
    """Serial (T < 64) and parallel-in-time Riccati both report a control
    weight that is not positive definite."""
    n, m = 2, 2
    A, B, Q, R, abar = _random_lqr(T, n, m, seed=1)
    cov.cov_lqr_track(ctx, dev64(A), dev64(B), Q, -np.eye(2), dev64(abar))
    st, fl = ctx.device_status()
    assert fl & (cov.DEV_NOT_SPD | cov.DEV_NONFINITE) and st == cov.COV_ERR_NONFINITE


def test_lqr_unicycle_long_horizon(cov, ctx, orc):
    """T = 65536 time-varying unicycle linearisation (the large workload's
    LQR), position-only weight, through the parallel-in-time Riccati."""
    T, dt = 65536, 0.01
    s0, u = wl.unicycle_init(T, dt)
    u = u + np.stack([0.05 * np.sin(np.arange(T) / 500.0), 0.5 * np.cos(np.arange(T) / 800.0)], 1)
    s = orc.rollout(wl.UNICYCLE, s0, u, dt)
    A, B = orc.linearize(wl.UNICYCLE, s, u, dt)
    abar = np.zeros((T, 3))
    abar[:, :2] = wl.rng(7).standard_normal((T, 2)) * 0.05
    Q, R = wl.coverage_Q(wl.UNICYCLE), 0.01 * np.eye(2)
    v, z = cov.cov_lqr_track(ctx, dev64(A), dev64(B), Q, R, dev64(abar))
    vo, zo, _ = orc.lqr_track(A, B, Q, R, abar)
    np.testing.assert_allclose(host(v), vo, rtol=1e-8, atol=1e-10 * np.abs(vo).max())
    np.testing.assert_allclose(host(z), zo, rtol=1e-8, atol=1e-10 * np.abs(zo).max())
    assert ctx.device_status()[1] == 0


@pytest.mark.parametrize("T", [1, 255, 256, 257, 513, 1024, 1025, 4096, 10001])
@pytest.mark.parametrize("model", [wl.SINGLE_INT, wl.DOUBLE_INT, wl.UNICYCLE])
def test_linearize_and_rollout_match_oracle(cov, ctx, orc, model, T):
    """Up to 256 steps the rollout is one CTA's block scans; longer horizons
    chunk its sums over the GPU (256 steps per chunk, the state entering
    each chunk from the earlier chunks' totals): T spans one chunk, its
    edge, several chunks and a ragged last one."""
    n, m = wl.MODEL_DIMS[model]
    dt = 0.03
    g = wl.rng(model)
    s0 = g.standard_normal(n)
    u = g.standard_normal((T, m))
    s = cov.cov_rollout(ctx, model, s0, dev64(u), dt)
    so = orc.rollout(model, s0, u, dt)
    np.testing.assert_allclose(host(s), so, rtol=1e-12, atol=1e-12)
    A, B = cov.cov_linearize(ctx, model, dev64(so), dev64(u), dt)
    Ao, Bo = orc.linearize(model, so, u, dt)
    np.testing.assert_allclose(host(A), Ao, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(host(B), Bo, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("T", [1, 100, 256, 512, 513])
def test_single_integrator_fused_step_matches_oracle(cov, ctx, orc, T):
    """Up to T = 512 the single integrator's LQR step, control update and
    rollout run as one launch (the short kernel with the update fused; T =
    513 takes the separate kernels): one outer iteration of the Stein field
    against the oracle's, controls and trajectory, and two more outer
    iterations on the same context (cached gains and short-kernel matrices)."""
    w = dataclasses.replace(wl.SVGD_SINGLE_T256, name="svgd_fused_check", T=T, dt=0.1 * 256 / max(T, 100), n_outer=1)
    inst = wl.make_instance(w)
    gmm = tuple(wl.f32_pair(v)[1] for v in inst.gmm)
    prob = cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, gmm=gmm, h=w.h)
    s_init = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    u = dev64(inst.u0)
    s = cov.cov_solve(ctx, prob, 1, u)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    uo, so = orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, 1, gmm=gmm, h=w.h)
    assert rel_norm(host(s) - s_init, so - s_init) <= 1e-4
    assert rel_norm(host(u) - inst.u0, uo - inst.u0) <= 1e-4
    np.testing.assert_array_equal(host(s)[0], inst.s0)
    # the new trajectory is the rollout of the new controls
    np.testing.assert_allclose(host(s), orc.rollout(w.model, inst.s0, host(u), w.dt), rtol=0, atol=1e-12)
    cov.cov_solve_continue(ctx, prob, 2, u, s)
    assert ctx.device_status()[0] == cov.COV_OK
    uo3, so3 = orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, 3, gmm=gmm, h=w.h)
    assert rel_norm(host(s) - s_init, so3 - s_init) <= 1e-4
    np.testing.assert_allclose(host(s), orc.rollout(w.model, inst.s0, host(u), w.dt), rtol=0, atol=1e-12)


@pytest.mark.parametrize("model", [wl.SINGLE_INT, wl.DOUBLE_INT, wl.UNICYCLE])
def test_rollout_update_in_solve_matches_oracle(cov, ctx, orc, model):
    """The update u += eta v fused into the chunked rollout (the cov_solve
    path, T = 1000 > one chunk): one outer iteration of the Stein field
    against the oracle's, controls and trajectory."""
    w = dataclasses.replace(wl.SVGD_SINGLE_T256, name="svgd_rollout_check", model=model, T=1000, dt=0.01,
                            n_outer=1)
    inst = wl.make_instance(w)
    gmm = tuple(wl.f32_pair(v)[1] for v in inst.gmm)
    prob = cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, gmm=gmm, h=w.h)
    u = dev64(inst.u0)
    s = cov.cov_solve(ctx, prob, 1, u)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    uo, so = orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, 1, gmm=gmm, h=w.h)
    s_init = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    # the step is eta * z(field); FP32 field error bounds its relative error
    assert rel_norm(host(s) - s_init, so - s_init) <= 1e-4
    assert rel_norm(host(u) - inst.u0, uo - inst.u0) <= 1e-4
