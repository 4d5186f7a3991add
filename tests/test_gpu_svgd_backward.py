"""Gradients through K outer iterations of a Stein-field solve (Eq. 4,
Sec. II-C) with a Gaussian-mixture reference: cov_solve_backward_svgd
against the FP64 oracle's reverse sweep (itself pinned by central
differences), teacher-forced with the GPU's own checkpoints, and the
autograd wrapper against central differences of the oracle's forward solve.

Bars: 1e-4 norm-wise for a few outer iterations (the field's bar); 1e-3
through the 100 outer iterations of the Stein workload, where the reverse
sweep adds the FP32 rounding of 100 field reverse passes; for the
directional derivative |g . v - FD| <= 2e-3 |g| (the end-to-end bar)."""
import numpy as np
import pytest
import torch

from conftest import dev64, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problem(cov, model, T, dt, s0, gmm, h, Q, R, eta):
    return cov.make_problem(model, T, dt, s0, wl.FIELD_SVGD, Q, R, eta, gmm=gmm, h=h)


@pytest.mark.parametrize("model,T,K", [(wl.DOUBLE_INT, 300, 3), (wl.SINGLE_INT, 513, 2)])
def test_reverse_sweep_matches_oracle_teacher_forced(cov, ctx, orc, model, T, K):
    dt, h, eta = 0.05, 0.08, 0.01
    n, m = wl.MODEL_DIMS[model]
    gmm = tuple(wl.f32_pair(v)[1] for v in wl.gmm_params(5, seed=91))
    if model == wl.SINGLE_INT:
        s0, u0 = wl.line_controls_single(T, dt, seed=92)
    else:
        s0, u0 = wl.double_int_init(T, dt)
    Q, R = wl.coverage_Q(model), 0.05 * np.eye(m)
    P = _problem(cov, model, T, dt, s0, gmm, h, Q, R, eta)
    u = dev64(u0)
    s_K, hist = cov.cov_solve_checkpointed(ctx, P, K, u)
    c = wl.rng(93).standard_normal((T + 1, n))
    got = cov.cov_solve_backward_svgd(ctx, P, K, dev64(u0), dev64(c), s_hist=hist)
    rep = cov.cov_solve_backward_svgd(ctx, P, K, dev64(u0), dev64(c))
    assert ctx.device_status() == (cov.COV_OK, 0)
    for a, b in zip(got, rep):  # replayed checkpoints are the same trajectories
        np.testing.assert_array_equal(host(a), host(b))
    want = orc.solve_backward_svgd(model, dt, 2, gmm, h, Q, R, eta, host(hist)[:K], c)
    for a, b in zip(got, want):
        assert rel_norm(host(a), b) <= 1e-4


def test_stein_workload_reverse_sweep_through_100_outer_iterations(cov, ctx, orc):
    """The Stein workload at full size: single integrator, T = 256, 3-component
    mixture, h = 0.05, 100 outer iterations."""
    inst = wl.make_instance(wl.SVGD_SINGLE_T256)
    w = inst.wl
    gmm = tuple(wl.f32_pair(v)[1] for v in inst.gmm)
    P = _problem(cov, w.model, w.T, w.dt, inst.s0, gmm, w.h, inst.Q, inst.R, w.eta)
    s_K, hist = cov.cov_solve_checkpointed(ctx, P, w.n_outer, dev64(inst.u0))
    c = wl.rng(94).standard_normal((w.T + 1, 2))
    got = cov.cov_solve_backward_svgd(ctx, P, w.n_outer, dev64(inst.u0), dev64(c), s_hist=hist)
    assert ctx.device_status() == (cov.COV_OK, 0)
    want = orc.solve_backward_svgd(w.model, w.dt, 2, gmm, w.h, inst.Q, inst.R, w.eta, host(hist), c)
    for a, b in zip(got, want):
        assert rel_norm(host(a), b) <= 1e-3


def test_autograd_directional_derivative_against_oracle_forward(cov, orc):
    """CoverageSolveStein on the Stein workload (T = 256, 100 outer
    iterations): the gradient of L = <c, s^K> with respect to the mixture
    (3 weights, 6 mean coordinates, 3 standard deviations) and s_0, along a
    random unit direction, against the central difference (step 1e-6) of
    two FP64 oracle solves."""
    from paper_2511_11514_b300 import autograd as ag
    inst = wl.make_instance(wl.SVGD_SINGLE_T256)
    w = inst.wl
    gw, gmu, gsig = (wl.f32_pair(v)[1] for v in inst.gmm)
    c = wl.rng(95).standard_normal((w.T + 1, 2))
    ctx = cov.Context(0)
    try:
        tw = torch.tensor(gw, dtype=torch.float32, requires_grad=True)
        tm = torch.tensor(gmu, dtype=torch.float32, requires_grad=True)
        ts = torch.tensor(gsig, dtype=torch.float32, requires_grad=True)
        t0 = torch.tensor(inst.s0, dtype=torch.float64, requires_grad=True)
        spec = dict(model=w.model, dt=w.dt, Q=inst.Q, R=inst.R, eta=w.eta, h=w.h, n_outer=w.n_outer)
        s_K = ag.CoverageSolveStein.apply(tw, tm, ts, t0, dev64(inst.u0), spec, ctx)
        (torch.as_tensor(c, device="cuda") * s_K).sum().backward()
        assert ctx.device_status() == (cov.COV_OK, 0)
        g = np.concatenate([tw.grad.double().numpy(), tm.grad.double().numpy().ravel(),
                            ts.grad.double().numpy(), t0.grad.numpy()])
    finally:
        ctx.close()
    theta = np.concatenate([gw, gmu.ravel(), gsig, np.asarray(inst.s0, dtype=np.float64)])

    def L(th):
        gm = (th[:3], th[3:9].reshape(3, 2), th[9:12])
        _, s = orc.solve(w.model, w.dt, th[12:14], inst.u0, w.field, inst.Q, inst.R, w.eta, w.n_outer, gmm=gm,
                         h=w.h)
        return float(np.sum(c * s))

    v = wl.rng(96).standard_normal(theta.size)
    v /= np.linalg.norm(v)
    fd = (L(theta + 1e-6 * v) - L(theta - 1e-6 * v)) / 2e-6
    assert abs(float(g @ v) - fd) <= 2e-3 * np.linalg.norm(g), (float(g @ v), fd, np.linalg.norm(g))
