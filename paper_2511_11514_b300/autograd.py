"""Differentiable coverage synthesis on the libcov adjoint (torch.autograd).

Four pieces, each a thin ``torch.autograd.Function`` over C-ABI calls (the
forward and backward arithmetic runs in libcov's kernels), or input
reparameterisation:

* ``CoverageSolve``: the final trajectory s^K after K outer iterations of
  Sec. II-C (Sinkhorn field, time-invariant model) as a function of the
  reference samples y, their weights b and the initial state s0.  Forward:
  ``cov_solve_checkpointed`` keeps the trajectory entering every outer
  iteration; backward: ``cov_solve_backward`` runs the reverse sweep (rollout,
  LQR and field adjoints) from those checkpoints.
* ``CoverageSolveStein``: the same for the Stein field (Eq. 4) with a
  Gaussian-mixture reference, as a function of the mixture's weights, means
  and standard deviations and the initial state (``cov_solve_backward_svgd``).
* ``SinkhornLoss``: the debiased Sinkhorn divergence of Eq. 6 between the
  samples x and a held-out reference set (uniform weights).  Give it a
  context of its own: a field call on the solve's context overwrites the
  time-invariant Riccati gains that cov_solve caches in its workspace (they
  are then recomputed).  ``cov_sinkhorn_divergence`` computes the value, the
  dual value <a, f> + <b, g> - <a, p> - <b, q> at the potentials after
  n_iter iterations, and the gradient, the envelope formula -(1/T) times
  the field of Eq. 7 at those potentials (exact at convergence).
* ``gmm_reference``: reference samples and weights of a Gaussian mixture by
  reparameterisation, y_j = mu_c + sigma_c xi_j (M/K fixed standard normal
  draws per component c) and b_j = softmax(logits)_c / (M/K), in plain torch
  ops so that autograd carries dL/dy, dL/db to the mixture parameters.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as cov


class CoverageSolve(torch.autograd.Function):
    """s_K = CoverageSolve.apply(y, b, s0, u0, spec, ctx).

    y [M, d] float32 CUDA, b [M] float32 CUDA or None, s0 [n] float64,
    u0 [T, m] float64 CUDA (not differentiated through by autograd's graph
    unless it requires grad: its gradient dL/du0 is returned too).
    spec: dict(model, dt, Q, R, eta, eps, n_iter, n_outer).  The forward keeps
    every outer iteration's Sinkhorn record in the workspace and the backward
    reuses it when no other forward ran on the context in between (else it
    recomputes from the saved checkpoints); both replay cached CUDA graphs.
    Returns s^K [T+1, n] float64 CUDA."""

    @staticmethod
    def forward(fctx, y, b, s0, u0, spec, cctx):
        T, m = u0.shape
        s0h = s0.detach().cpu().double().numpy()
        P = cov.make_problem(spec["model"], T, spec["dt"], s0h, cov.FIELD_SINKHORN, spec["Q"], spec["R"],
                             spec["eta"], d=y.shape[1], y=y.detach(), b=None if b is None else b.detach(),
                             eps=spec["eps"], n_iter=spec["n_iter"])
        s_K, hist, token, P = cov.grad_forward(cctx, P, spec["n_outer"], u0.detach(), y.detach(),
                                               None if b is None else b.detach())
        fctx.problem = P
        fctx.cctx = cctx
        fctx.n_outer = spec["n_outer"]
        fctx.token = token
        fctx.has_b = b is not None
        fctx.s0_meta = (s0.device, s0.dtype)
        fctx.save_for_backward(u0.detach(), hist, y.detach(), None if b is None else b.detach())
        return s_K

    @staticmethod
    def backward(fctx, g_K):
        u0, hist, y, b = fctx.saved_tensors
        ybar, bbar, s0bar, u0bar = cov.grad_backward(fctx.cctx, fctx.problem, fctx.n_outer, u0,
                                                     g_K.detach().double().contiguous(), hist, fctx.token, y, b)
        dev, dt = fctx.s0_meta
        return (ybar, bbar if fctx.has_b else None, s0bar.to(device=dev, dtype=dt), u0bar, None, None)


class CoverageSolveStein(torch.autograd.Function):
    """s_K = CoverageSolveStein.apply(w, mu, sigma, s0, u0, spec, ctx): the
    final trajectory after K outer iterations of a Stein-field solve (Eq. 4,
    Sec. II-C) with the Gaussian-mixture reference (w [K] raw weights, mu
    [K, d], sigma [K]; any device, float) on a time-invariant model, as a
    function of the mixture and the initial state s0 [n] (float64).
    spec: dict(model, dt, Q, R, eta, h, n_outer).  The forward keeps the
    trajectory entering every outer iteration (cov_solve_checkpointed); the
    backward runs cov_solve_backward_svgd from those checkpoints.  Returns
    s^K [T+1, n] float64 CUDA; the gradient for u0 [T, m] is returned too."""

    @staticmethod
    def forward(fctx, w, mu, sigma, s0, u0, spec, cctx):
        T, m = u0.shape
        d = mu.shape[1]
        gmm = tuple(v.detach().cpu().float().numpy() for v in (w, mu, sigma))
        P = cov.make_problem(spec["model"], T, spec["dt"], s0.detach().cpu().double().numpy(), cov.FIELD_SVGD,
                             spec["Q"], spec["R"], spec["eta"], d=d, gmm=gmm, h=spec["h"])
        u = u0.detach().clone().contiguous()
        s_K, hist = cov.cov_solve_checkpointed(cctx, P, spec["n_outer"], u)
        fctx.problem = P
        fctx.cctx = cctx
        fctx.n_outer = spec["n_outer"]
        fctx.meta = [(v.device, v.dtype) for v in (w, mu, sigma, s0)]
        fctx.save_for_backward(u0.detach(), hist)
        return s_K

    @staticmethod
    def backward(fctx, g_K):
        u0, hist = fctx.saved_tensors
        wb, mb, sb, s0b, u0b = cov.cov_solve_backward_svgd(fctx.cctx, fctx.problem, fctx.n_outer, u0,
                                                           g_K.detach().double().contiguous(), s_hist=hist)
        out = [t.to(device=dv, dtype=dt) for t, (dv, dt) in zip((wb, mb, sb, s0b), fctx.meta)]
        return (*out, u0b, None, None)


class SinkhornLoss(torch.autograd.Function):
    """L = SinkhornLoss.apply(x, y_ref, eps, n_iter, cctx, q_ref): S_eps of the
    uniform sample sets x [T, d] and y_ref [M, d] (float32 CUDA), computed by
    ``cov_sinkhorn_divergence`` (value and gradient in the library); q_ref is
    the reference's self potential from ``reference_self_potential`` (or
    None: recomputed by every call)."""

    @staticmethod
    def forward(fctx, x, y_ref, eps, n_iter, cctx, q_ref=None):
        value, grad, _ = cov.cov_sinkhorn_divergence(cctx, x.detach().contiguous(), y_ref, eps, n_iter,
                                                     q_ref=q_ref, q_given=q_ref is not None)
        fctx.save_for_backward(grad)
        return value

    @staticmethod
    def backward(fctx, gL):
        (grad,) = fctx.saved_tensors
        return (gL.to(grad.dtype) * grad, None, None, None, None, None)


def reference_self_potential(cctx, y_ref, eps, n_iter):
    """Self potential q [M] of the uniform set y_ref after n_iter averaged
    self updates (the p output of a field evaluation of y_ref against
    itself), for SinkhornLoss's q_ref."""
    _, _, _, q = cov.cov_field_sinkhorn(cctx, y_ref, y_ref, eps, n_iter, field=False)
    return q


def gmm_reference(mu, log_sigma, logits, xi):
    """(y [M, d], b [M]) of the mixture by reparameterisation: component c
    owns the rows c*M/K .. (c+1)*M/K - 1 of the fixed draws xi [M, d]."""
    K = mu.shape[0]
    M, d = xi.shape
    per = M // K
    if per * K != M:
        raise ValueError("M must be a multiple of the number of components")
    # broadcast over the per-component blocks (a gather's backward would be a
    # scatter-add; this one is a plain reduction)
    y = (mu[:, None, :] + torch.exp(log_sigma)[:, None, None] * xi.view(K, per, d)).reshape(M, d)
    b = (torch.softmax(logits, 0)[:, None] / per).expand(K, per).reshape(M)
    return y.float().contiguous(), b.float().contiguous()


def standard_draws(M: int, d: int, seed: int, device="cuda"):
    """Fixed standard normal draws xi [M, d] (seeded, float32-exact)."""
    g = np.random.Generator(np.random.Philox(seed))
    return torch.as_tensor(g.standard_normal((M, d)).astype(np.float32), device=device)
