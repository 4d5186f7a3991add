"""GPU parity of the Sinkhorn variants (eps-scaling within a field
evaluation, warm-started potentials across outer iterations) against the
oracle's definitions of the same schedules.

Bars as for the plain field: potentials max|f_gpu - f_orc|/eps <= 1e-4,
fields norm-wise 1e-4; the warm solve's trajectory displacement 1e-4."""
import numpy as np
import pytest
import torch

from conftest import dev32, dev64, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu

POT_TOL = 1e-4
FIELD_TOL = 1e-4


@pytest.mark.parametrize("T,M,eps,n_iter,e0,dec,weighted", [
    (300, 517, 0.005, 30, 0.08, 0.8, True),
    (1000, 2100, 0.002, 40, 0.05, 0.85, False),
    (257, 129, 0.01, 5, 0.2, 0.5, True),      # ends before reaching eps: the last step rescales to eps
    (64, 64, 0.01, 6, 0.005, 0.5, False),     # eps_start below eps: the plain iteration
])
def test_annealed_field_matches_oracle(cov, ctx, orc, T, M, eps, n_iter, e0, dec, weighted):
    x = wl.random_points(T, 2, seed=701)
    y = wl.random_points(M, 2, seed=702)
    b = wl.random_weights(M, seed=703) if weighted else None
    a, f, g, p = cov.cov_field_sinkhorn_annealed(ctx, dev32(x), dev32(y), eps, n_iter, e0, dec,
                                                 b=dev32(b) if weighted else None)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    fo, go, po = orc.sinkhorn_annealed(x, y, b, eps, n_iter, e0, dec)
    ao = orc.sinkhorn_field(x, y, b, eps, go, po)
    for u, v in ((f, fo), (g, go), (p, po)):
        assert np.abs(host(u) - v).max() / eps <= POT_TOL
    assert rel_norm(host(a), ao) <= FIELD_TOL


def test_annealed_field_with_warm_start(cov, ctx, orc):
    T, M, eps = 400, 600, 0.004
    x = wl.random_points(T, 2, seed=711)
    y = wl.random_points(M, 2, seed=712)
    f0, g0, p0 = orc.sinkhorn(x + 0.01, y, None, eps, 20)        # potentials of a nearby problem
    f0, g0, p0 = (wl.f32_pair(v)[1] for v in (f0, g0, p0))
    a, f, g, p = cov.cov_field_sinkhorn_annealed(ctx, dev32(x), dev32(y), eps, 12, 0.03, 0.7, f=dev32(f0),
                                                 g=dev32(g0), p=dev32(p0), warm=True)
    fo, go, po = orc.sinkhorn_annealed(x, y, None, eps, 12, 0.03, 0.7, f=f0, g=g0, p=p0)
    for u, v in ((f, fo), (g, go), (p, po)):
        assert np.abs(host(u) - v).max() / eps <= POT_TOL
    assert rel_norm(host(a), orc.sinkhorn_field(x, y, None, eps, go, po)) <= FIELD_TOL


@pytest.mark.parametrize("use_graph", [0, 1])
def test_warm_solve_matches_oracle(cov, ctx, orc, use_graph):
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=256, M=512)
    w = inst.wl
    eps, n_iter, K = 0.02, 8, 3
    P = cov.make_problem(w.model, 256, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, y=dev32(inst.y), eps=eps,
                         n_iter=n_iter, warm=True, eps_start=0.1, eps_decay=0.7)
    ctx.set_option(cov.OPT_USE_GRAPH, use_graph)
    try:
        u = dev64(inst.u0)
        s = cov.cov_solve(ctx, P, K, u)
    finally:
        ctx.set_option(cov.OPT_USE_GRAPH, 1)
    uo, so = orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, K, y=inst.y, eps=eps,
                       n_iter=n_iter, warm=True, eps_start=0.1, eps_decay=0.7)
    s_init = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    assert rel_norm(host(s) - s_init, so - s_init) <= 1e-4
    assert rel_norm(host(u) - inst.u0, uo - inst.u0) <= 1e-4


def test_warm_continuation_is_one_solve(cov, ctx):
    """cov_solve(2) then cov_solve_continue(1) keeps the potentials and
    equals cov_solve(3) bit for bit."""
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=300, M=400)
    w = inst.wl
    P = cov.make_problem(w.model, 300, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, y=dev32(inst.y), eps=0.02,
                         n_iter=6, warm=True)
    u1 = dev64(inst.u0)
    s1 = cov.cov_solve(ctx, P, 2, u1)
    cov.cov_solve_continue(ctx, P, 1, u1, s1)
    u2 = dev64(inst.u0)
    s2 = cov.cov_solve(ctx, P, 3, u2)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    np.testing.assert_array_equal(host(s1), host(s2))


def test_backward_rejects_the_variants(cov, ctx):
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=128, M=128)
    w = inst.wl
    for kw in (dict(warm=True), dict(eps_start=0.1, eps_decay=0.5)):
        P = cov.make_problem(w.model, 128, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, y=dev32(inst.y),
                             eps=0.02, n_iter=4, **kw)
        with pytest.raises(cov.CovError):
            cov.cov_solve_backward(ctx, P, 1, dev64(inst.u0), torch.zeros((129, 4), dtype=torch.float64,
                                                                          device="cuda"))


def test_invalid_decay_is_rejected(cov, ctx):
    x = dev32(wl.random_points(16, 2, seed=1))
    with pytest.raises(cov.CovError):
        cov.cov_field_sinkhorn_annealed(ctx, x, x, 0.01, 3, 0.1, 1.5)


# -- Stein field with a pixel-density reference --------------------------------------
DENSITY_TOL = 1e-4   # norm-wise; FP32 cell coordinate u = x W - 1/2 resolves 2^-24 W of a pixel


def test_density_score_matches_oracle(cov, ctx, orc):
    m = wl.f32_pair(wl.density_map(seed=3))[1]
    x = wl.random_points(20000, 2, seed=801, lo=-0.05, hi=1.05)   # includes the clamped border strip
    sc = cov.cov_density_score(ctx, dev32(m), dev32(x))
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    so = orc.density_score(m, x)
    assert rel_norm(host(sc), so) <= DENSITY_TOL


@pytest.mark.parametrize("use_graph", [0, 1])
def test_svgd_solve_with_density_matches_oracle(cov, ctx, orc, use_graph):
    inst = wl.make_instance(wl.SVGD_SINGLE_T256)
    w = inst.wl
    m = wl.f32_pair(wl.density_map(seed=4, n=128))[1]
    eta = 1e-3
    P = cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, eta, density=dev32(m), h=w.h)
    ctx.set_option(cov.OPT_USE_GRAPH, use_graph)
    try:
        u = dev64(inst.u0)
        s = cov.cov_solve(ctx, P, 3, u)
    finally:
        ctx.set_option(cov.OPT_USE_GRAPH, 1)
    uo, so = orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, eta, 3, h=w.h, density=m)
    s_init = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    assert rel_norm(host(s) - s_init, so - s_init) <= 1e-4


# -- fixed-offset updates: the overflow and underflow fallbacks -----------------------
_CONVERGED = {}


def _converged(orc, T, M, eps):
    """Points, weights and 30-iteration potentials of one seeded problem."""
    key = (T, M, eps)
    if key not in _CONVERGED:
        x = wl.random_points(T, 2, seed=721)
        y = wl.random_points(M, 2, seed=722)
        b = wl.random_weights(M, seed=723)
        _CONVERGED[key] = (x, y, b) + orc.sinkhorn(x, y, b, eps, 30)
    return _CONVERGED[key]


@pytest.mark.parametrize("T,M", [(300, 517), (3000, 5000)])
@pytest.mark.parametrize("which,shift", [("g", 0.8), ("g", 5.0), ("f", 0.8)])
@pytest.mark.parametrize("n_iter", [1, 5])
def test_warm_offsets_far_from_the_update(cov, ctx, orc, T, M, which, shift, n_iter):
    """Warm-started updates take the log-sum-exp implied by the given
    potentials as their fixed row offset.  Per-row shifts of the given g (or
    f) by -shift, 0 or +shift move that offset by shift / (eps ln 2) bits
    (115 bits for 0.8 at eps = 0.01, 721 for 5.0) from the update's own
    log-sum-exp: some rows' fixed-offset sums overflow (above 2^100, finite or
    infinite: the CTA redoes its columns with a running maximum), others
    underflow (below 2^-60, or zero: the row block is recomputed over all
    columns).  The given g enters only the offsets, so with shifted g the
    result is the unshifted warm start's; in both cases it is the oracle's
    warm-started iteration, whose arithmetic has no offsets."""
    eps = 0.01
    x, y, b, fc, gc, pc = _converged(orc, T, M, eps)
    rng = wl.rng(724)
    if which == "g":
        gc = gc + shift * rng.integers(-1, 2, size=M)
    else:
        fc = fc + shift * rng.integers(-1, 2, size=T)
    f0, g0, p0 = (wl.f32_pair(v)[1] for v in (fc, gc, pc))
    a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(x), dev32(y), eps, n_iter, b=dev32(b), f=dev32(f0), g=dev32(g0),
                                        p=dev32(p0), warm=True)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    fo, go, po = orc.sinkhorn(x, y, b, eps, n_iter, f=f0, g=g0, p=p0)
    for u, v in ((f, fo), (g, go), (p, po)):
        assert np.abs(host(u) - v).max() / eps <= POT_TOL
    assert rel_norm(host(a), orc.sinkhorn_field(x, y, b, eps, go, po)) <= FIELD_TOL
