"""Batched solve (one CUDA graph per outer iteration for many problems):
every problem's result must equal the same problem solved alone."""
import dataclasses

import numpy as np
import pytest
import torch

from conftest import dev32, dev64, host
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problem(cov, inst, ydev):
    w = inst.wl
    if w.field == wl.FIELD_SVGD:
        return cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, gmm=inst.gmm, h=w.h)
    return cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, y=ydev, eps=w.eps,
                            n_iter=w.n_iter)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_batch_equals_problems_solved_alone(cov, ctx, use_graph):
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
    try:
        us = [dev64(i.u0) for i in insts]
        ss = cov.cov_solve_batched(ctx, probs, n_outer, us)
        torch.cuda.synchronize()
        for i, pr, ub, sb in zip(insts, probs, us, ss):
            u1 = dev64(i.u0)
            s1 = cov.cov_solve(ctx, pr, n_outer, u1)
            np.testing.assert_array_equal(host(sb), host(s1))
            np.testing.assert_array_equal(host(ub), host(u1))
    finally:
        ctx.set_option(cov.OPT_USE_GRAPH, 1)
    assert ctx.device_status() == (cov.COV_OK, 0)


def test_batch_rejects_bad_problem(cov, ctx):
    insts = wl.make_batch(3, seed=4, T_range=(40, 60), M_range=(50, 80), K_range=(2, 3))
    ys = [dev32(i.y) if i.y is not None else None for i in insts]
    probs = [_problem(cov, i, y) for i, y in zip(insts, ys)]
    probs[1][0].eta = float("nan")
    with pytest.raises(cov.CovError):
        cov.cov_solve_batched(ctx, probs, 1, [dev64(i.u0) for i in insts])
