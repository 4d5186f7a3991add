"""GPU outer iteration (Sec. II-C) against the oracle: one iteration on
identical inputs, and final coverage metric within 1% after many
iterations (trajectories are not compared after many iterations: the
problem has many equally good optima)."""
import numpy as np
import pytest
import torch

from conftest import dev32, dev64, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problem(cov, inst, T, n_iter=None, eps=None, y_dev=None):
    w = inst.wl
    if w.field == wl.FIELD_SVGD:
        return cov.make_problem(w.model, T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, gmm=inst.gmm, h=w.h)
    return cov.make_problem(w.model, T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, y=y_dev,
                            eps=w.eps if eps is None else eps, n_iter=w.n_iter if n_iter is None else n_iter)


def _metric(orc, s, ref):
    return orc.sinkhorn_divergence(s[1:, :2], ref, None, 0.01, tol=1e-7)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_svgd_solve_one_iteration(cov, ctx, orc, use_graph):
    inst = wl.make_instance(wl.SVGD_SINGLE_T256)
    w = inst.wl
    gmm = tuple(wl.f32_pair(v)[1] for v in inst.gmm)
    inst.gmm = gmm
    ctx.set_option(cov.OPT_USE_GRAPH, use_graph)
    try:
        u = dev64(inst.u0)
        s = cov.cov_solve(ctx, _problem(cov, inst, w.T), 1, u)
    finally:
        ctx.set_option(cov.OPT_USE_GRAPH, 1)
    uo, so = orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, 1, gmm=gmm, h=w.h)
    s_init = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    # the step is eta * z(field); FP32 field error bounds its relative error
    assert rel_norm(host(s) - s_init, so - s_init) <= 1e-4
    assert rel_norm(host(u) - inst.u0, uo - inst.u0) <= 1e-4


def test_sinkhorn_solve_one_iteration(cov, ctx, orc):
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=512, M=1024)
    w = inst.wl
    u = dev64(inst.u0)
    s = cov.cov_solve(ctx, _problem(cov, inst, 512, n_iter=10, y_dev=dev32(inst.y)), 1, u)
    uo, so = orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, 1, y=inst.y,
                       eps=w.eps, n_iter=10)
    s_init = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    assert rel_norm(host(s) - s_init, so - s_init) <= 1e-4


def test_svgd_solve_final_metric_within_one_percent(cov, ctx, orc):
    """The SVGD single-integrator workload at full size: T = 256, 100 outer
    iterations, against the oracle's own solve."""
    inst = wl.make_instance(wl.SVGD_SINGLE_T256)
    w = inst.wl
    inst.gmm = tuple(wl.f32_pair(v)[1] for v in inst.gmm)
    u = dev64(inst.u0)
    s = cov.cov_solve(ctx, _problem(cov, inst, w.T), w.n_outer, u)
    uo, so = orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, w.n_outer,
                       gmm=inst.gmm, h=w.h)
    ref = wl.f32_pair(wl.gmm_samples(*inst.gmm, 1 << 10, seed=1))[1]
    mg, mo = _metric(orc, host(s), ref), _metric(orc, so, ref)
    m0 = _metric(orc, orc.rollout(w.model, inst.s0, inst.u0, w.dt), ref)
    assert mo < m0
    assert abs(mg - mo) <= 0.01 * abs(mo)


def test_sinkhorn_solve_final_metric_within_one_percent(cov, ctx, orc):
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=384, M=1024)
    w = inst.wl
    n_outer, n_iter = 30, 20
    u = dev64(inst.u0)
    s = cov.cov_solve(ctx, _problem(cov, inst, 384, n_iter=n_iter, y_dev=dev32(inst.y)), n_outer, u)
    uo, so = orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, n_outer, y=inst.y,
                       eps=w.eps, n_iter=n_iter)
    ref = wl.f32_pair(wl.gmm_samples(*inst.gmm, 1 << 10, seed=1))[1]
    mg, mo = _metric(orc, host(s), ref), _metric(orc, so, ref)
    assert abs(mg - mo) <= 0.01 * abs(mo)
    assert ctx.device_status()[1] == 0


def test_cached_gains_survive_other_calls_on_the_context(cov, ctx):
    """cov_solve caches the Riccati gains of a time-invariant model in the
    workspace; a field call in between overwrites that scratch, so the next
    cov_solve_continue must recompute them: solving 2 + 2 iterations around a
    foreign field call equals solving 4 in one call, bit for bit."""
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=512, M=1024)
    P = _problem(cov, inst, 512, n_iter=10, y_dev=dev32(inst.y))
    u1 = dev64(inst.u0)
    s1 = cov.cov_solve(ctx, P, 2, u1)
    xo = dev32(wl.random_points(3000, 2, seed=5))
    cov.cov_field_sinkhorn(ctx, xo, dev32(wl.random_points(5000, 2, seed=6)), 0.003, 7)
    cov.cov_solve_continue(ctx, P, 2, u1, s1)
    u2 = dev64(inst.u0)
    s2 = cov.cov_solve(ctx, P, 4, u2)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    np.testing.assert_array_equal(host(s1), host(s2))
    np.testing.assert_array_equal(host(u1), host(u2))
