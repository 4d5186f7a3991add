"""GPU parity of the adjoints against the FP64 oracle adjoints.

The field VJP differentiates the FP32 forward iterations exactly, so its
difference from the oracle is the FP32 rounding of the recorded potentials
carried through the reverse sweep; it is judged norm-wise (FIELD_VJP_TOL).
The LQR and rollout adjoints run in FP64 and must agree to reassociation
level.  The full backward is compared teacher-forced: the oracle's reverse
sweep is given the GPU forward's checkpoints and the same dL/ds^K.  At the
full differentiation workload (T = 2048, M = 8192, 50 iterations, 20 outer
iterations) the oracle is too slow, so two exact identities are checked
instead: translating the reference set and the initial position together
moves the final trajectory rigidly, and scaling all weights changes nothing.
"""
import numpy as np
import pytest
import torch

from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELD_VJP_TOL = 1e-4   # norm-wise, FP32 reverse sweep vs FP64 oracle (measured <= 1.1e-5)
FP64_TOL = 1e-9


def _dev32(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _dev64(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _h(t):
    return t.detach().cpu().double().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("T,M,d,eps,n_iter,weighted", [
    (300, 517, 2, 0.02, 5, True),
    (700, 1100, 2, 0.005, 12, False),
    (257, 300, 3, 0.05, 3, True),
    (150, 200, 1, 0.02, 4, True),
    (130, 70, 2, 0.01, 0, True),       # no iteration: the field of the cold potentials
    (1, 9, 2, 0.05, 2, True),          # a single sample
])
def test_field_vjp_matches_oracle(cov, ctx, orc, T, M, d, eps, n_iter, weighted):
    x = wl.random_points(T, d, seed=201)
    y = wl.random_points(M, d, seed=202)
    b = wl.random_weights(M, seed=203) if weighted else None
    abar = wl.f32_pair(wl.rng(204).standard_normal((T, d)))[1]
    xg, yg, bg = cov.cov_field_sinkhorn_vjp(ctx, _dev32(x), _dev32(y), eps, n_iter, _dev32(abar),
                                            b=_dev32(b) if weighted else None)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    xo, yo, bo = orc.sinkhorn_field_vjp(x, y, b, eps, n_iter, abar)
    ex, ey = _rel(_h(xg), xo), _rel(_h(yg), yo)
    assert ex <= FIELD_VJP_TOL, ex
    assert ey <= FIELD_VJP_TOL, ey
    if weighted:
        eb = _rel(_h(bg), bo)
        assert eb <= FIELD_VJP_TOL, eb
    else:
        assert bg is None


def test_field_vjp_translation_and_scale_identities(cov, ctx):
    """Exact at any size: a common translation of x and y leaves the field
    unchanged (sum xbar + sum ybar = 0), and so does scaling all weights
    (sum_j b_j bbar_j = 0)."""
    T, M, d, eps, n_iter = 2048, 8192, 2, 0.005, 50
    x = wl.random_points(T, d, seed=211, lo=0.1, hi=0.9)
    y = wl.random_points(M, d, seed=212)
    b = wl.random_weights(M, seed=213)
    abar = wl.f32_pair(wl.rng(214).standard_normal((T, d)))[1]
    xg, yg, bg = cov.cov_field_sinkhorn_vjp(ctx, _dev32(x), _dev32(y), eps, n_iter, _dev32(abar), b=_dev32(b))
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    xs, ys = _h(xg).sum(0), _h(yg).sum(0)
    scale = np.abs(_h(xg)).sum(0) + np.abs(_h(yg)).sum(0)
    assert np.all(np.abs(xs + ys) <= 1e-3 * scale), (xs, ys, scale)
    bb = _h(bg) * b
    assert abs(bb.sum()) <= 1e-3 * np.abs(bb).sum()


@pytest.mark.parametrize("T,n,m", [(1, 2, 2), (37, 4, 2), (600, 4, 2), (300, 3, 2), (129, 4, 3)])
def test_lqr_vjp_matches_oracle(cov, ctx, orc, T, n, m):
    r = wl.rng(300 + T)
    A = np.stack([0.97 * np.linalg.qr(r.standard_normal((n, n)))[0] for _ in range(T)])
    B = 0.3 * r.standard_normal((T, n, m))
    L = r.standard_normal((n, n))
    Q = L @ L.T + 0.5 * np.eye(n)
    R = 0.1 * np.eye(m)
    vbar = r.standard_normal((T, m))
    got = _h(cov.cov_lqr_vjp(ctx, _dev64(A), _dev64(B), Q, R, _dev64(vbar)))
    want = orc.lqr_vjp(A, B, Q, R, vbar)
    assert _rel(got, want) <= FP64_TOL


@pytest.mark.parametrize("model", [wl.SINGLE_INT, wl.DOUBLE_INT, wl.UNICYCLE])
def test_rollout_vjp_matches_oracle(cov, ctx, orc, model):
    n, m = wl.MODEL_DIMS[model]
    T, dt = 1500, 0.02
    r = wl.rng(400 + model)
    s0 = np.concatenate([[0.2, 0.3], 0.3 * r.standard_normal(n - 2)])
    u = r.standard_normal((T, m))
    s = orc.rollout(model, s0, u, dt)
    sbar = r.standard_normal((T + 1, n))
    ug, s0g = cov.cov_rollout_vjp(ctx, model, _dev64(s), _dev64(u), dt, _dev64(sbar))
    uo, s0o = orc.rollout_vjp(model, s, u, dt, sbar)
    assert _rel(_h(ug), uo) <= FP64_TOL
    assert _rel(_h(s0g), s0o) <= FP64_TOL


def _problem(cov, inst):
    w = inst.wl
    y = _dev32(inst.y)
    b = _dev32(wl.random_weights(inst.y.shape[0], seed=77))
    P = cov.make_problem(w.model, inst.u0.shape[0], w.dt, inst.s0, wl.FIELD_SINKHORN, inst.Q, inst.R, w.eta, d=2,
                         y=y, b=b, eps=w.eps * 4, n_iter=8)
    return P, y, b


def test_solve_backward_matches_oracle_teacher_forced(cov, ctx, orc):
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=200, M=300)
    w = inst.wl
    K = 3
    (P, keep), y, b = _problem(cov, inst)
    u = _dev64(inst.u0)
    u0 = u.clone()
    s_K, hist = cov.cov_solve_checkpointed(ctx, (P, keep), K, u)
    sbar = wl.rng(501).standard_normal((inst.u0.shape[0] + 1, 4))
    yb, bb, s0b, u0b = cov.cov_solve_backward(ctx, (P, keep), K, u0, _dev64(sbar), s_hist=hist)
    yr, br, s0r, u0r = cov.cov_solve_backward(ctx, (P, keep), K, u0, _dev64(sbar))
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    # replaying the forward gives the same checkpoints, hence the same gradient
    np.testing.assert_array_equal(_h(yb), _h(yr))
    np.testing.assert_array_equal(_h(s0b), _h(s0r))
    yo, bo, s0o, u0o = orc.solve_backward(w.model, w.dt, 2, inst.y.astype(np.float64), _h(b), P.eps, P.n_iter,
                                          inst.Q, inst.R, w.eta, _h(hist)[:K], sbar)
    for got, want in ((yb, yo), (bb, bo), (s0b, s0o), (u0b, u0o)):
        assert _rel(_h(got), want) <= FIELD_VJP_TOL, (_rel(_h(got), want))


def test_solve_backward_translation_identity_at_full_size(cov, ctx):
    """T = 2048, M = 8192, 50 iterations, K = 20: translating y and the
    initial position by tau moves s^K rigidly by tau, so
    sum_j ybar_j + s0bar[:2] = sum_t sbar_K[t, :2]; and sum_j b_j bbar_j = 0."""
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=2048, M=8192)
    w = inst.wl
    K = 20
    y = _dev32(inst.y)
    bh = wl.random_weights(8192, seed=78)
    b = _dev32(bh)
    P, keep = cov.make_problem(w.model, 2048, w.dt, inst.s0, wl.FIELD_SINKHORN, inst.Q, inst.R, w.eta, d=2,
                               y=y, b=b, eps=w.eps, n_iter=50)
    u = _dev64(inst.u0)
    u0 = u.clone()
    s_K, hist = cov.cov_solve_checkpointed(ctx, (P, keep), K, u)
    sbar = wl.rng(502).standard_normal((2048 + 1, 4))
    yb, bb, s0b, u0b = cov.cov_solve_backward(ctx, (P, keep), K, u0, _dev64(sbar), s_hist=hist)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    lhs = _h(yb).sum(0) + _h(s0b)[:2]
    rhs = sbar[1:, :2].sum(0) + sbar[0, :2]
    assert np.all(np.abs(lhs - rhs) <= 2e-3 * (np.abs(rhs) + np.abs(_h(yb)).sum(0))), (lhs, rhs)
    wb = _h(bb) * bh
    assert abs(wb.sum()) <= 1e-3 * np.abs(wb).sum()
    assert np.isfinite(_h(u0b)).all()


def test_recorded_forward_gives_the_recomputed_gradient(cov, ctx):
    """A recording forward keeps every outer iteration's Sinkhorn record; the
    backward then skips the recomputation and must give, bit for bit, the
    gradient that recomputing from the same checkpoints gives.  The recorded
    forward itself follows cov_solve to FP32 rounding."""
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=700, M=900)
    K = 4
    (P, keep), y, b = _problem(cov, inst)
    u_rec = _dev64(inst.u0)
    s_rec, hist = cov.cov_solve_checkpointed(ctx, (P, keep), K, u_rec, record=True)
    sbar = _dev64(wl.rng(503).standard_normal((inst.u0.shape[0] + 1, 4)))
    u0 = _dev64(inst.u0)
    g_rec = cov.cov_solve_backward(ctx, (P, keep), K, u0, sbar, s_hist=hist)
    g_rec2 = cov.cov_solve_backward(ctx, (P, keep), K, u0, sbar, s_hist=hist)  # records still valid
    hist2 = hist.clone()  # another pointer: the records do not apply, the backward recomputes
    g_cmp = cov.cov_solve_backward(ctx, (P, keep), K, u0, sbar, s_hist=hist2)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    for a, a2, c in zip(g_rec, g_rec2, g_cmp):
        np.testing.assert_array_equal(_h(a), _h(c))
        np.testing.assert_array_equal(_h(a2), _h(c))
    u_pl = _dev64(inst.u0)
    s_pl = cov.cov_solve(ctx, (P, keep), K, u_pl)
    s_init = _h(hist[0])
    assert _rel(_h(s_rec) - s_init, _h(s_pl) - s_init) <= 1e-4
