"""torch.autograd over the libcov adjoint, end to end against the oracle.

The GPU gradient of the coverage loss (Sinkhorn divergence of the final
positions to a held-out set) through K outer iterations is compared with the
oracle's FP64 gradient (itself pinned by central differences).  Unlike the
teacher-forced test of the reverse sweep, each side runs its own forward
here, so the tolerance also covers the FP32 field's effect on the
trajectory and the finite iteration count of the GPU loss (the oracle
converges it to 1e-12).
"""
import numpy as np
import pytest
import torch

from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu

E2E_TOL = 2e-3


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_autograd_gradient_matches_oracle(cov, ctx, orc):
    from paper_2511_11514_b300 import autograd as ag
    T, M, ML, dt, K = 160, 200, 240, 0.05, 3
    s0h, u0h = wl.double_int_init(T, dt)
    yh = wl.random_points(M, 2, seed=601, lo=0.2, hi=0.8)
    bh = wl.random_weights(M, seed=602)
    ylh = wl.random_points(ML, 2, seed=603, lo=0.1, hi=0.9)
    Q = wl.coverage_Q(wl.DOUBLE_INT)
    R = 0.05 * np.eye(2)
    eps, n_iter, eta, eps_l, it_l = 0.05, 6, 0.5, 0.05, 400
    dev = torch.device("cuda")
    y = torch.tensor(yh, dtype=torch.float32, device=dev, requires_grad=True)
    b = torch.tensor(bh, dtype=torch.float32, device=dev, requires_grad=True)
    s0 = torch.tensor(s0h, dtype=torch.float64, requires_grad=True)
    u0 = torch.as_tensor(u0h, dtype=torch.float64, device=dev)
    y_loss = torch.as_tensor(ylh, dtype=torch.float32, device=dev)
    spec = dict(model=wl.DOUBLE_INT, dt=dt, Q=Q, R=R, eta=eta, eps=eps, n_iter=n_iter, n_outer=K)
    q_ref = ag.reference_self_potential(ctx, y_loss, eps_l, it_l)
    s_K = ag.CoverageSolve.apply(y, b, s0, u0, spec, ctx)
    L = ag.SinkhornLoss.apply(s_K[1:, :2].float().contiguous(), y_loss, eps_l, it_l, ctx, q_ref)
    L.backward()
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    Lo, yo, bo, s0o = orc.solve_sinkhorn_grad(wl.DOUBLE_INT, dt, s0h, u0h, 2, yh, bh, eps, n_iter, Q, R, eta, K,
                                              ylh, None, eps_l)
    assert float(L.detach()) == pytest.approx(Lo, rel=2e-3)
    assert _rel(y.grad.double().cpu().numpy(), yo) <= E2E_TOL
    assert _rel(b.grad.double().cpu().numpy(), bo) <= E2E_TOL
    assert _rel(s0.grad.numpy(), s0o) <= E2E_TOL


def test_reparameterised_mixture_gradients_are_the_chain_rule(cov, ctx):
    """Mixture parameters -> samples by reparameterisation: autograd's mean
    gradient equals the per-component sum of the sample gradients."""
    from paper_2511_11514_b300 import autograd as ag
    T, M, dt, K = 128, 256, 0.05, 2
    s0h, u0h = wl.double_int_init(T, dt)
    dev = torch.device("cuda")
    mu = torch.tensor([[0.3, 0.3], [0.6, 0.7], [0.4, 0.7], [0.7, 0.3]], dtype=torch.float32, device=dev,
                      requires_grad=True)
    log_sigma = torch.full((4,), float(np.log(0.08)), dtype=torch.float32, device=dev, requires_grad=True)
    logits = torch.zeros(4, dtype=torch.float32, device=dev, requires_grad=True)
    xi = ag.standard_draws(M, 2, seed=7, device=dev)
    y, b = ag.gmm_reference(mu, log_sigma, logits, xi)
    y.retain_grad()
    b.retain_grad()
    spec = dict(model=wl.DOUBLE_INT, dt=dt, Q=wl.coverage_Q(wl.DOUBLE_INT), R=0.05 * np.eye(2), eta=0.5, eps=0.05,
                n_iter=5, n_outer=K)
    y_loss = torch.as_tensor(wl.random_points(200, 2, seed=8), dtype=torch.float32, device=dev)
    s_K = ag.CoverageSolve.apply(y, b, torch.tensor(s0h), torch.as_tensor(u0h, device=dev), spec, ctx)
    L = ag.SinkhornLoss.apply(s_K[1:, :2].float().contiguous(), y_loss, 0.05, 200, ctx, None)
    L.backward()
    per = M // 4
    gy = y.grad.view(4, per, 2).sum(1)
    torch.testing.assert_close(mu.grad, gy, rtol=1e-5, atol=1e-6)
    assert torch.isfinite(log_sigma.grad).all() and torch.isfinite(logits.grad).all()
    # softmax weights: the logits gradient sums to zero (shift invariance)
    assert abs(float(logits.grad.sum())) <= 1e-5 * float(logits.grad.abs().sum() + 1e-12)


def test_interleaved_forwards_fall_back_to_recomputation(cov, ctx):
    """Two forwards, then the first one's backward: the records on the
    context belong to the second forward, so the first backward must
    recompute its Sinkhorn iterations -- and give the gradient a plain
    forward/backward pair gives."""
    from paper_2511_11514_b300 import autograd as ag
    T, M, dt, K = 256, 300, 0.05, 2
    s0h, u0h = wl.double_int_init(T, dt)
    dev = torch.device("cuda")
    spec = dict(model=wl.DOUBLE_INT, dt=dt, Q=wl.coverage_Q(wl.DOUBLE_INT), R=0.05 * np.eye(2), eta=0.5, eps=0.05,
                n_iter=5, n_outer=K)
    u0 = torch.as_tensor(u0h, device=dev)
    y_a = torch.tensor(wl.random_points(M, 2, seed=11), dtype=torch.float32, device=dev, requires_grad=True)
    y_b = torch.tensor(wl.random_points(M, 2, seed=12), dtype=torch.float32, device=dev, requires_grad=True)
    y_ref = torch.tensor(y_a.detach().cpu().numpy(), dtype=torch.float32, device=dev, requires_grad=True)
    w = torch.as_tensor(wl.random_points(T + 1, 4, seed=13), device=dev)

    def loss(y):
        return (ag.CoverageSolve.apply(y, None, torch.tensor(s0h), u0, spec, ctx) * w).sum()

    loss(y_ref).backward()           # forward + backward with the records
    La = loss(y_a)
    Lb = loss(y_b)                   # overwrites the records
    La.backward()                    # recomputes
    Lb.backward()                    # uses the records
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    torch.testing.assert_close(y_a.grad, y_ref.grad, rtol=0, atol=0)
    assert torch.isfinite(y_b.grad).all()


def test_full_size_directional_derivative_against_oracle_forward(cov, orc):
    """The differentiation workload at full size (T = 2048, M = 8192 samples
    of a 4-component mixture by reparameterisation, 50 iterations, K = 20
    outer iterations): the GPU gradient of L = <c, s^K> (c a fixed random
    cotangent of the final trajectory) with respect to the 20 parameters
    (means, log-sigmas, weight logits, s_0), taken along a random unit
    direction v, against the central difference (step 1e-6) of the FP64
    oracle's forward L(theta +- 1e-6 v).  A linear functional of s^K keeps
    the comparison on the reverse sweep through the 20 outer iterations
    (the Sinkhorn-loss gradient itself is the envelope formula, checked
    against the oracle in the divergence tests).  Bar: |g . v - FD| <=
    2e-3 |g| (Cauchy-Schwarz from the end-to-end gradient bar; with 20
    parameters a wrong gradient component moves g . v by ~|g| / 4.5)."""
    from paper_2511_11514_b300 import autograd as ag
    w = wl.ADJOINT_DOUBLE_T2048
    inst = wl.make_instance(w)
    gw, gmu, gsig = inst.gmm
    dev = torch.device("cuda", 0)
    xi = ag.standard_draws(w.M, 2, seed=w.seed + 2000, device=dev)
    xih = xi.double().cpu().numpy()
    c = wl.rng(901).standard_normal((w.T + 1, 4))
    theta0 = np.concatenate([np.asarray(gmu, dtype=np.float32).ravel(),
                             np.log(np.asarray(gsig, dtype=np.float32)).astype(np.float32),
                             np.log(np.asarray(gw, dtype=np.float32)).astype(np.float32),
                             np.asarray(inst.s0)]).astype(np.float64)
    theta0[:16] = theta0[:16].astype(np.float32).astype(np.float64)

    def split(th):
        return th[:8].reshape(4, 2), th[8:12], th[12:16], th[16:20]

    ctx = cov.Context(0)
    try:
        mu_t, ls_t, lg_t, s0_t = split(theta0)
        mu = torch.tensor(mu_t, dtype=torch.float32, device=dev, requires_grad=True)
        ls = torch.tensor(ls_t, dtype=torch.float32, device=dev, requires_grad=True)
        lg = torch.tensor(lg_t, dtype=torch.float32, device=dev, requires_grad=True)
        s0 = torch.tensor(s0_t, dtype=torch.float64, requires_grad=True)
        spec = dict(model=w.model, dt=w.dt, Q=inst.Q, R=inst.R, eta=w.eta, eps=w.eps, n_iter=w.n_iter,
                    n_outer=w.n_outer)
        y, b = ag.gmm_reference(mu, ls, lg, xi)
        s_K = ag.CoverageSolve.apply(y, b, s0, torch.as_tensor(inst.u0, device=dev), spec, ctx)
        L = (torch.as_tensor(c, device=dev) * s_K).sum()
        L.backward()
        st, flags = ctx.device_status()
        assert st == cov.COV_OK, flags
        g = np.concatenate([mu.grad.double().cpu().numpy().ravel(), ls.grad.double().cpu().numpy(),
                            lg.grad.double().cpu().numpy(), s0.grad.numpy()])
    finally:
        ctx.close()

    def oracle_loss(th):
        m, lsig, logit, s0v = split(th)
        per = w.M // 4
        yv = (m[:, None, :] + np.exp(lsig)[:, None, None] * xih.reshape(4, per, 2)).reshape(w.M, 2)
        pw = np.exp(logit - logit.max())
        bv = np.repeat(pw / pw.sum() / per, per)
        _, s = orc.solve(w.model, w.dt, s0v, inst.u0, wl.FIELD_SINKHORN, inst.Q, inst.R, w.eta, w.n_outer,
                         y=yv, b=bv, eps=w.eps, n_iter=w.n_iter)
        return float(np.sum(c * s))

    v = wl.rng(902).standard_normal(20)
    v /= np.linalg.norm(v)
    hstep = 1e-6
    fd = (oracle_loss(theta0 + hstep * v) - oracle_loss(theta0 - hstep * v)) / (2 * hstep)
    dd = float(g @ v)
    assert abs(dd - fd) <= 2e-3 * np.linalg.norm(g), (dd, fd, np.linalg.norm(g))
