"""Batched solve (one CUDA graph per outer iteration for many problems):
every problem's result must equal the same problem solved alone."""
import dataclasses

import numpy as np
import pytest
import torch

from conftest import dev32, dev64, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu



def _problem(cov, inst, ydev):
    w = inst.wl
    if w.field == wl.FIELD_SVGD:
        return cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, gmm=inst.gmm, h=w.h)
    return cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, y=ydev, eps=w.eps,
                            n_iter=w.n_iter)


@pytest.mark.parametrize("use_graph,share", [(1, 100), (0, 100), (1, 0)])
def test_batch_equals_problems_solved_alone(cov, ctx, use_graph, share):
    """With every problem's launches planned for the whole GPU (share 100)
    the batch runs exactly the single-problem kernels and plans, so each
    problem's result equals cov_solve on it alone, bit for bit.  With the
    default planning share the column splits differ, so the sums are taken
    in another order: then the trajectories agree to FP32 rounding of the
    field (1e-5 of the displacement)."""
    insts = wl.make_batch(7, seed=3, T_range=(37, 700), M_range=(50, 1500), K_range=(2, 5))
    for i in insts:
        if i.wl.field == wl.FIELD_SINKHORN:
            i.wl.n_iter = 8
    # one unicycle problem in the mix (time-varying Riccati inside the graph)
    u_inst = wl.make_instance(wl.SINKHORN_UNICYCLE_T65536, T=300, M=400)
    u_inst.wl = dataclasses.replace(u_inst.wl, T=300, M=400, n_iter=6)
    insts.append(u_inst)
    ys = [dev32(i.y) if i.y is not None else None for i in insts]
    probs = [_problem(cov, i, y) for i, y in zip(insts, ys)]
    n_outer = 3
    ctx.set_option(cov.OPT_USE_GRAPH, use_graph)
    if share:
        ctx.set_option(cov.OPT_BATCH_SHARE, share)
    try:
        us = [dev64(i.u0) for i in insts]
        ss = cov.cov_solve_batched(ctx, probs, n_outer, us)
        torch.cuda.synchronize()
        for i, pr, ub, sb in zip(insts, probs, us, ss):
            u1 = dev64(i.u0)
            s1 = cov.cov_solve(ctx, pr, n_outer, u1)
            if share == 100:
                np.testing.assert_array_equal(host(sb), host(s1))
                np.testing.assert_array_equal(host(ub), host(u1))
            else:
                s_init = host(cov.cov_rollout(ctx, i.wl.model, i.s0, dev64(i.u0), i.wl.dt))
                assert rel_norm(host(sb) - s_init, host(s1) - s_init) <= 1e-5
    finally:
        ctx.set_option(cov.OPT_USE_GRAPH, 1)
        ctx.set_option(cov.OPT_BATCH_SHARE, cov.BATCH_SHARE_DEFAULT)
    assert ctx.device_status() == (cov.COV_OK, 0)


def test_batch_rejects_bad_problem(cov, ctx):
    insts = wl.make_batch(3, seed=4, T_range=(40, 60), M_range=(50, 80), K_range=(2, 3))
    ys = [dev32(i.y) if i.y is not None else None for i in insts]
    probs = [_problem(cov, i, y) for i, y in zip(insts, ys)]
    probs[1][0].eta = float("nan")
    with pytest.raises(cov.CovError):
        cov.cov_solve_batched(ctx, probs, 1, [dev64(i.u0) for i in insts])


def _oracle_one_iteration(orc, inst):
    w = inst.wl
    if w.field == wl.FIELD_SVGD:
        return orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, 1, gmm=inst.gmm, h=w.h)
    return orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, 1, y=inst.y, eps=w.eps,
                     n_iter=w.n_iter)


def _check_against_oracle(orc, inst, s_gpu, u_gpu, tol):
    """One outer iteration from the same initial controls on both sides: the
    trajectory moves by the rollout of eta v*(field), so its displacement and
    the control change are compared norm-wise (Sec. II-C; the field bar of
    1e-4 carries over to v*, which is linear in the field)."""
    w = inst.wl
    uo, so = _oracle_one_iteration(orc, inst)
    s_init = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    es = rel_norm(host(s_gpu) - s_init, so - s_init)
    eu = rel_norm(host(u_gpu) - inst.u0, uo - inst.u0)
    assert es <= tol and eu <= tol, (w.name, w.field, w.T, w.M, es, eu)


def test_batch_one_iteration_matches_oracle(cov, ctx, orc):
    """A mixed batch (Stein and Sinkhorn fields on the double integrator, one
    unicycle problem with a time-varying Riccati) solved for one outer
    iteration in one graph launch: every problem against the FP64 oracle's
    own solve of it."""
    insts = wl.make_batch(6, seed=5, T_range=(60, 900), M_range=(100, 2000), K_range=(2, 16))
    for i in insts:
        if i.wl.field == wl.FIELD_SINKHORN:
            i.wl.n_iter = 12
    u_inst = wl.make_instance(wl.SINKHORN_UNICYCLE_T65536, T=333, M=500)
    u_inst.wl = dataclasses.replace(u_inst.wl, T=333, M=500, n_iter=10)
    insts.append(u_inst)
    ys = [dev32(i.y) if i.y is not None else None for i in insts]
    probs = [_problem(cov, i, y) for i, y in zip(insts, ys)]
    us = [dev64(i.u0) for i in insts]
    ss = cov.cov_solve_batched(ctx, probs, 1, us)
    torch.cuda.synchronize()
    assert ctx.device_status() == (cov.COV_OK, 0)
    for i, ub, sb in zip(insts, us, ss):
        _check_against_oracle(orc, i, sb, ub, 1e-4)


def test_full_shape_batch_of_1024_problems_against_oracle(cov, ctx, orc):
    """The batched workload at full shape: 1024 double-integrator problems,
    T ~ U{128..4096}, M ~ U{512..16384}, 2-16 component mixtures, half Stein
    and half Sinkhorn (eps = 0.005, 50 iterations), one outer iteration of all
    of them in one graph launch; the first and the longest Stein problem (the
    one-launch Stein field and, past T = 1024, the all-pairs one), the
    smallest and the largest Sinkhorn problem are checked against the FP64
    oracle."""
    insts = wl.make_batch(1024)
    ys = [dev32(i.y) if i.y is not None else None for i in insts]
    probs = [_problem(cov, i, y) for i, y in zip(insts, ys)]
    c = cov.Context(0)
    try:
        us = [dev64(i.u0) for i in insts]
        ss = cov.cov_solve_batched(c, probs, 1, us)
        torch.cuda.synchronize()
        assert c.device_status() == (cov.COV_OK, 0)
        sk = [k for k, i in enumerate(insts) if i.wl.field == wl.FIELD_SINKHORN]
        cost = {k: insts[k].wl.T * (insts[k].wl.M + insts[k].wl.T) for k in sk}
        sv = [k for k, i in enumerate(insts) if i.wl.field == wl.FIELD_SVGD]
        picks = [sv[0], max(sv, key=lambda k: insts[k].wl.T), min(sk, key=cost.get), max(sk, key=cost.get)]
        for k in picks:
            _check_against_oracle(orc, insts[k], ss[k], us[k], 1e-4)
    finally:
        c.close()
