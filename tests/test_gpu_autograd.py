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
    assert float(L) == pytest.approx(Lo, rel=2e-3)
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
