"""Pins of the oracle's reverse-mode adjoints (gradients through the outer
iteration of Sec. II-C).

Independent references: central finite differences of the forward oracle
functions along random directions (every input perturbed separately, so a
wrong term in one input's gradient cannot be hidden by another), and, for the
LQR adjoint, the transpose of a dense KKT solve built with numpy plus the
dot-product identity <vbar, v(abar)> = <abar, vjp(vbar)> of a linear map.
"""
import numpy as np
import pytest

from paper_2511_11514_b300 import workloads as wl

from test_oracle_lqr import _dense_kkt

H = 1e-6


def _field_obj(orc, x, y, b, eps, n_iter, abar):
    f, g, p = orc.sinkhorn(x, y, b, eps, n_iter)
    return float(np.sum(abar * orc.sinkhorn_field(x, y, b, eps, g, p)))


def _fd(fun, base, direction, h=H):
    return (fun(base + h * direction) - fun(base - h * direction)) / (2 * h)


@pytest.mark.parametrize("T,M,d,eps,n_iter,weighted", [
    (9, 13, 2, 0.05, 0, True),      # zero potentials: the field of the plain softmax barycentres
    (9, 13, 2, 0.05, 1, False),
    (11, 17, 2, 0.02, 6, True),
    (7, 10, 3, 0.1, 4, True),
])
def test_field_vjp_matches_central_differences(orc, T, M, d, eps, n_iter, weighted):
    x = wl.random_points(T, d, seed=31)
    y = wl.random_points(M, d, seed=32)
    b = wl.random_weights(M, seed=33) if weighted else None
    r = wl.rng(34)
    abar = r.standard_normal((T, d))
    xbar, ybar, bbar = orc.sinkhorn_field_vjp(x, y, b, eps, n_iter, abar)
    scale = max(np.abs(xbar).max(), np.abs(ybar).max(), 1.0)

    dx = r.standard_normal((T, d))
    fd = _fd(lambda xx: _field_obj(orc, xx, y, b, eps, n_iter, abar), x, dx)
    assert np.sum(xbar * dx) == pytest.approx(fd, rel=1e-6, abs=1e-7 * scale)

    dy = r.standard_normal((M, d))
    fd = _fd(lambda yy: _field_obj(orc, x, yy, b, eps, n_iter, abar), y, dy)
    assert np.sum(ybar * dy) == pytest.approx(fd, rel=1e-6, abs=1e-7 * scale)

    if weighted:
        db = r.standard_normal(M) * b          # relative perturbation keeps b > 0
        fd = _fd(lambda bb: _field_obj(orc, x, y, bb, eps, n_iter, abar), b, db)
        assert np.sum(bbar * db) == pytest.approx(fd, rel=1e-6, abs=1e-7 * scale)
        # scaling all weights leaves the normalised measure, hence the field, unchanged
        assert np.sum(bbar * b) == pytest.approx(0.0, abs=1e-9 * np.abs(bbar * b).sum())


def test_field_vjp_single_coordinates(orc):
    """Every coordinate of x and y separately on a tiny case (catches a
    transposed index that a random direction could average away)."""
    T, M, d, eps, n_iter = 4, 5, 2, 0.08, 3
    x = wl.random_points(T, d, seed=41)
    y = wl.random_points(M, d, seed=42)
    abar = wl.rng(43).standard_normal((T, d))
    xbar, ybar, _ = orc.sinkhorn_field_vjp(x, y, None, eps, n_iter, abar)
    for arr, grad, which in ((x, xbar, 0), (y, ybar, 1)):
        for i in range(arr.shape[0]):
            for c in range(d):
                e = np.zeros_like(arr)
                e[i, c] = 1.0
                if which == 0:
                    fd = _fd(lambda xx: _field_obj(orc, xx, y, None, eps, n_iter, abar), x, e)
                else:
                    fd = _fd(lambda yy: _field_obj(orc, x, yy, None, eps, n_iter, abar), y, e)
                assert grad[i, c] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def _lqr_case(T, n, m, seed, time_varying):
    r = wl.rng(seed)
    if time_varying:
        A = np.stack([0.97 * np.linalg.qr(r.standard_normal((n, n)))[0] for _ in range(T)])
    else:
        A = np.broadcast_to(np.eye(n) + 0.05 * r.standard_normal((n, n)), (T, n, n)).copy()
    B = r.standard_normal((T, n, m)) * 0.3
    L = r.standard_normal((n, n))
    Q = L @ L.T + 0.5 * np.eye(n)
    Rm = 0.1 * np.eye(m) + 0.01 * np.diag(r.random(m))
    return A, B, Q, Rm


@pytest.mark.parametrize("T,n,m,tv", [(1, 2, 2, False), (6, 3, 2, True), (30, 4, 2, False),
                                      (25, 4, 3, True)])
def test_lqr_vjp_is_transpose_of_dense_kkt(orc, T, n, m, tv):
    A, B, Q, Rm = _lqr_case(T, n, m, 50 + T, tv)
    r = wl.rng(60 + T)
    vbar = r.standard_normal((T, m))
    got = orc.lqr_vjp(A, B, Q, Rm, vbar)
    # dense: v = H^-1 G'Qb abar  =>  abar_bar = Qb G H^-1 vbar
    Gm = np.zeros((T * n, T * m))
    for s in range(T):
        blk = B[s]
        for t in range(s + 1, T + 1):
            Gm[(t - 1) * n:t * n, s * m:(s + 1) * m] = blk
            if t < T:
                blk = A[t] @ blk
    Qb = np.kron(np.eye(T), Q)
    Hm = Gm.T @ Qb @ Gm + np.kron(np.eye(T), Rm)
    want = (Qb @ Gm @ np.linalg.solve(Hm, vbar.reshape(-1))).reshape(T, n)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-10 * np.abs(want).max())
    # the same through the forward oracle: <vbar, v(abar)> = <abar, vjp(vbar)>
    abar = r.standard_normal((T, n))
    v, _, _ = orc.lqr_track(A, B, Q, Rm, abar)
    vd, _ = _dense_kkt(A, B, Q, Rm, abar)
    np.testing.assert_allclose(v, vd, rtol=1e-9, atol=1e-11)
    assert np.sum(vbar * v) == pytest.approx(np.sum(abar * got), rel=1e-10)


@pytest.mark.parametrize("model", [wl.SINGLE_INT, wl.DOUBLE_INT, wl.UNICYCLE])
def test_rollout_vjp_matches_central_differences(orc, model):
    n, m = wl.MODEL_DIMS[model]
    T, dt = 15, 0.05
    r = wl.rng(70 + model)
    s0 = np.concatenate([[0.2, 0.3], 0.3 * r.standard_normal(n - 2)])
    u = r.standard_normal((T, m))
    s = orc.rollout(model, s0, u, dt)
    sbar = r.standard_normal((T + 1, n))
    ubar, s0bar = orc.rollout_vjp(model, s, u, dt, sbar)
    obj_u = lambda uu: float(np.sum(sbar * orc.rollout(model, s0, uu, dt)))
    obj_s = lambda ss: float(np.sum(sbar * orc.rollout(model, ss, u, dt)))
    du = r.standard_normal(u.shape)
    assert np.sum(ubar * du) == pytest.approx(_fd(obj_u, u, du), rel=1e-7, abs=1e-9)
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        assert s0bar[c] == pytest.approx(_fd(obj_s, s0, e), rel=1e-7, abs=1e-9)


def _small_solve_case(model):
    n, m = wl.MODEL_DIMS[model]
    T, M, ML, dt = 20, 24, 30, 0.05
    if model == wl.DOUBLE_INT:
        s0, u0 = wl.double_int_init(T, dt)
    else:
        s0 = np.array([0.15, 0.2])
        u0 = np.tile([[0.6, 0.5]], (T, 1))
    y = wl.random_points(M, 2, seed=81, lo=0.2, hi=0.8)
    b = wl.random_weights(M, seed=82)
    yl = wl.random_points(ML, 2, seed=83, lo=0.1, hi=0.9)
    Q = wl.coverage_Q(model)
    Rm = 0.05 * np.eye(m)
    return dict(model=model, dt=dt, s0=s0, u0=u0, d=2, y=y, b=b, eps=0.05, n_iter=6, Q=Q, R=Rm,
                eta=0.5, n_outer=3, y_loss=yl, b_loss=None, eps_loss=0.05)


@pytest.mark.parametrize("model", [wl.SINGLE_INT, wl.DOUBLE_INT])
def test_solve_gradient_matches_central_differences(orc, model):
    """Loss after three outer iterations, differentiated with respect to the
    reference samples y, their weights b and the initial state s0."""
    kw = _small_solve_case(model)
    L, ybar, bbar, s0bar = orc.solve_sinkhorn_grad(**kw)
    assert L > 0.0
    r = wl.rng(90 + model)

    def loss(**over):
        k = dict(kw, **over)
        return orc.solve_sinkhorn_grad(**k)[0]

    dy = r.standard_normal(kw["y"].shape)
    fd = _fd(lambda yy: loss(y=yy), kw["y"], dy, h=1e-5)
    assert np.sum(ybar * dy) == pytest.approx(fd, rel=1e-5, abs=1e-9)
    db = r.standard_normal(kw["b"].shape) * kw["b"]
    fd = _fd(lambda bb: loss(b=bb), kw["b"], db, h=1e-5)
    assert np.sum(bbar * db) == pytest.approx(fd, rel=1e-5, abs=1e-9)
    for c in range(len(kw["s0"])):
        e = np.zeros(len(kw["s0"]))
        e[c] = 1.0
        fd = _fd(lambda ss: loss(s0=ss), kw["s0"], e, h=1e-5)
        assert s0bar[c] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_solve_gradient_rejects_trajectory_dependent_linearisation(orc):
    kw = _small_solve_case(wl.DOUBLE_INT)
    kw.update(model=wl.UNICYCLE, s0=np.array([0.1, 0.1, 0.3]), Q=wl.coverage_Q(wl.UNICYCLE))
    with pytest.raises(ValueError):
        orc.solve_sinkhorn_grad(**kw)


def test_backward_with_checkpoints_matches_central_differences_in_u0(orc):
    """The reverse sweep from explicit checkpoints: its u0 gradient of a
    linear functional of the final trajectory against central differences
    (two outer iterations, the functional <sbar, s^K>)."""
    kw = _small_solve_case(wl.DOUBLE_INT)
    K = 2
    r = wl.rng(99)
    sbar = r.standard_normal((kw["u0"].shape[0] + 1, 4))
    common = dict(d=2, y=kw["y"], b=kw["b"], eps=kw["eps"], n_iter=kw["n_iter"])
    hist = orc.solve_history(kw["model"], kw["dt"], kw["s0"], kw["u0"], kw["Q"], kw["R"], kw["eta"], K,
                             **common)
    ybar, bbar, s0bar, u0bar = orc.solve_backward(kw["model"], kw["dt"], 2, kw["y"], kw["b"], kw["eps"],
                                                  kw["n_iter"], kw["Q"], kw["R"], kw["eta"], hist[:K], sbar)

    def fun(u0=kw["u0"], y=kw["y"], s0=kw["s0"]):
        c = dict(common, y=y)
        h = orc.solve_history(kw["model"], kw["dt"], s0, u0, kw["Q"], kw["R"], kw["eta"], K, **c)
        return float(np.sum(sbar * h[-1]))

    du = r.standard_normal(kw["u0"].shape)
    assert np.sum(u0bar * du) == pytest.approx(_fd(lambda uu: fun(u0=uu), kw["u0"], du, h=1e-5), rel=1e-6)
    dy = r.standard_normal(kw["y"].shape)
    assert np.sum(ybar * dy) == pytest.approx(_fd(lambda yy: fun(y=yy), kw["y"], dy, h=1e-5), rel=1e-5)
    e = np.zeros(4)
    e[1] = 1.0
    assert s0bar[1] == pytest.approx(_fd(lambda ss: fun(s0=ss), kw["s0"], e, h=1e-5), rel=1e-6)


def _stein_history(orc, model, dt, s0, u0, gmm, h, Q, R, eta, K):
    """Checkpoints s^0..s^{K-1} and the final trajectory of a Stein solve."""
    u = np.array(u0, dtype=np.float64)
    hist = [orc.rollout(model, s0, u, dt)]
    for _ in range(K):
        u, s = orc.solve(model, dt, s0, u, wl.FIELD_SVGD, Q, R, eta, 1, gmm=gmm, h=h)
        hist.append(s)
    return np.stack(hist[:-1]), hist[-1]


@pytest.mark.parametrize("model", [wl.SINGLE_INT, wl.DOUBLE_INT])
def test_stein_solve_backward_matches_central_differences(orc, model):
    """<c, s^K> through K = 3 outer iterations of a Stein-field solve,
    differentiated by central differences along random directions in the
    mixture's raw weights, means and standard deviations, s_0 and u_0
    separately, against the oracle's reverse sweep."""
    T, K, dt, h, eta = 24, 3, 0.1, 0.12, 0.01
    n, m = wl.MODEL_DIMS[model]
    w, mu, sigma = wl.gmm_params(3, seed=81)
    if model == wl.SINGLE_INT:
        s0, u0 = wl.line_controls_single(T, dt, seed=82)
    else:
        s0, u0 = wl.double_int_init(T, dt)
    Q = wl.coverage_Q(model)
    R = 0.05 * np.eye(m)
    c = wl.rng(83).standard_normal((T + 1, n))

    def L(w_, mu_, sig_, s0_, u0_):
        _, sK = _stein_history(orc, model, dt, s0_, u0_, (w_, mu_, sig_), h, Q, R, eta, K)
        return float(np.sum(c * sK))

    hist, _ = _stein_history(orc, model, dt, s0, u0, (w, mu, sigma), h, Q, R, eta, K)
    wb, mb, sb, s0b, u0b = orc.solve_backward_svgd(model, dt, 2, (w, mu, sigma), h, Q, R, eta, hist, c)
    r = wl.rng(84)
    for grad, base, fun in ((wb, w, lambda v: L(v, mu, sigma, s0, u0)),
                            (mb, mu, lambda v: L(w, v, sigma, s0, u0)),
                            (sb, sigma, lambda v: L(w, mu, v, s0, u0)),
                            (s0b, np.asarray(s0, dtype=np.float64), lambda v: L(w, mu, sigma, v, u0)),
                            (u0b, np.asarray(u0, dtype=np.float64), lambda v: L(w, mu, sigma, s0, v))):
        dv = r.standard_normal(np.shape(base))
        fd = _fd(fun, np.asarray(base, dtype=np.float64), dv)
        assert float(np.sum(grad * dv)) == pytest.approx(fd, rel=1e-6, abs=1e-9)
    assert abs(float(np.dot(w, wb))) <= 1e-9 * float(np.abs(w * wb).sum())


def test_field_vjp_every_coordinate_at_64_by_128(orc):
    """Every coordinate of x (64 x 2), y (128 x 2) and b (128) separately by
    central differences (step 1e-6), at T = 64, M = 128 with 6 iterations:
    the all-coordinates check at a size where column splits and many rows
    matter."""
    T, M, d, eps, n_iter = 64, 128, 2, 0.05, 6
    x = wl.random_points(T, d, seed=51)
    y = wl.random_points(M, d, seed=52)
    b = wl.random_weights(M, seed=53)
    abar = wl.rng(54).standard_normal((T, d))
    xbar, ybar, bbar = orc.sinkhorn_field_vjp(x, y, b, eps, n_iter, abar)

    def fd_all(fun, base):
        g = np.zeros_like(base)
        for idx in np.ndindex(base.shape):
            e = np.zeros_like(base)
            e[idx] = 1.0
            g[idx] = _fd(fun, base, e)
        return g

    gx = fd_all(lambda v: _field_obj(orc, v, y, b, eps, n_iter, abar), x)
    gy = fd_all(lambda v: _field_obj(orc, x, v, b, eps, n_iter, abar), y)
    gb = fd_all(lambda v: _field_obj(orc, x, y, v, eps, n_iter, abar), b)
    np.testing.assert_allclose(xbar, gx, rtol=1e-5, atol=1e-6 * np.abs(gx).max())
    np.testing.assert_allclose(ybar, gy, rtol=1e-5, atol=1e-6 * np.abs(gy).max())
    np.testing.assert_allclose(bbar, gb, rtol=1e-5, atol=1e-6 * np.abs(gb).max())
