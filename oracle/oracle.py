"""ctypes binding of the FP64 CPU oracle (``cov_oracle.c``).

Test infrastructure only (see the package docstring).  All arrays are float64
numpy arrays, C-contiguous, row-major, shapes as documented per function.

Parity status per function:
  gmm_score, svgd_field, sinkhorn_*, sinkhorn_field, sinkhorn_divergence,
  linearize, rollout, lqr_track -- pinned (tests/test_oracle_*.py).
  sinkhorn_field_vjp, lqr_vjp, rollout_vjp, solve_backward, solve_sinkhorn_grad -- pinned by
  central finite differences of the forward functions and, for lqr_vjp, by
  the transpose identity against the dense KKT solve (tests/test_oracle_adjoint.py).
  solve -- composition of pinned parts; pinned only by the one-iteration
  composition check (single integrator, R -> 0: the trajectory moves by
  eta * field) and by the decrease of the coverage divergence.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cov_oracle.c")
_HDR = os.path.join(_HERE, "cov_oracle.h")
_LIB = os.path.join(_HERE, "libcov_oracle.so")

SINGLE_INT, DOUBLE_INT, UNICYCLE = 0, 1, 2
FIELD_SVGD, FIELD_SINKHORN = 0, 1
MODEL_DIMS = {SINGLE_INT: (2, 2), DOUBLE_INT: (4, 2), UNICYCLE: (3, 2)}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64, no fast-math)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-D_GNU_SOURCE", "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _declare(_lib)
    return _lib


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_i, _d = ctypes.c_int, ctypes.c_double


def _declare(L):
    sig = {
        "orc_set_threads": (None, [_i]),
        "orc_get_threads": (_i, []),
        "orc_gmm_logpdf": (_d, [_D, _i, _i, _D, _D, _D]),
        "orc_gmm_score": (None, [_D, _i, _i, _i, _D, _D, _D, _D]),
        "orc_svgd_field": (None, [_D, _i, _i, _D, _d, _I, _i, _D]),
        "orc_svgd_field_vjp": (None, [_D, _i, _i, _D, _d, _D, _D, _D]),
        "orc_gmm_score_vjp": (None, [_D, _i, _i, _i, _D, _D, _D, _D, _D, _D, _D, _D]),
        "orc_sinkhorn_g_update": (None, [_D, _i, _D, _i, _i, _d, _D, _I, _i, _D]),
        "orc_sinkhorn_f_update": (None, [_D, _i, _D, _i, _D, _i, _d, _D, _I, _i, _D]),
        "orc_sinkhorn_p_update": (None, [_D, _i, _i, _d, _D, _I, _i, _D]),
        "orc_sinkhorn": (None, [_D, _i, _D, _i, _D, _i, _d, _i, _i, _D, _D, _D]),
        "orc_sinkhorn_field": (None, [_D, _i, _D, _i, _D, _i, _d, _D, _D, _I, _i, _D]),
        "orc_sinkhorn_converge": (_i, [_D, _i, _D, _i, _D, _i, _d, _d, _i, _D, _D, _D]),
        "orc_sinkhorn_marginals": (None, [_D, _i, _D, _i, _D, _i, _d, _D, _D, _D, _D]),
        "orc_sinkhorn_divergence": (_d, [_D, _i, _D, _i, _D, _i, _d, _d, _i]),
        "orc_model_dims": (_i, [_i, _I, _I]),
        "orc_step": (None, [_i, _D, _D, _d, _D]),
        "orc_linearize": (None, [_i, _D, _D, _i, _d, _D, _D]),
        "orc_rollout": (None, [_i, _D, _D, _i, _d, _D]),
        "orc_lqr_track": (None, [_D, _D, _D, _D, _D, _i, _i, _i, _D, _D, _D]),
        "orc_solve": (_i, [_i, _i, _d, _D, _i, _i, _D, _D, _i, _i, _D, _D, _D,
                           _d, _i, _d, _D, _D, _d, _i, _D, _D]),
        "orc_anneal_eps": (_d, [_d, _d, _d, _i]),
        "orc_sinkhorn_annealed": (None, [_D, _i, _D, _i, _D, _i, _d, _i, _d, _d, _i, _D, _D, _D]),
        "orc_solve_ex": (_i, [_i, _i, _d, _D, _i, _i, _D, _D, _i, _i, _D, _D, _D,
                              _d, _i, _d, _D, _D, _d, _i, _D, _D, _i, _d, _d, _D, _i, _i]),
        "orc_density_value": (_d, [_D, _i, _i, _D]),
        "orc_density_score": (None, [_D, _i, _i, _D, _i, _D]),
        "orc_sinkhorn_field_vjp": (None, [_D, _i, _D, _i, _D, _i, _d, _i, _D, _D, _D, _D]),
        "orc_lqr_vjp": (None, [_D, _D, _D, _D, _D, _i, _i, _i, _D]),
        "orc_rollout_vjp": (None, [_i, _D, _D, _i, _d, _D, _D, _D]),
        "orc_solve_backward": (_i, [_i, _i, _d, _i, _D, _D, _i, _d, _i, _D, _D, _d, _i, _D, _D,
                                    _D, _D, _D, _D]),
        "orc_solve_backward_svgd": (_i, [_i, _i, _d, _i, _i, _D, _D, _D, _d, _D, _D, _d, _i, _D, _D, _D, _D, _D,
                                         _D, _D]),
        "orc_solve_sinkhorn_grad": (_d, [_i, _i, _d, _D, _i, _D, _D, _i, _d, _i, _D, _D, _d, _i,
                                         _D, _D, _D, _i, _d, _D, _D, _D]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def _rows(rows):
    if rows is None:
        return None, None, 0
    r = np.ascontiguousarray(rows, dtype=np.int32)
    return r, r.ctypes.data_as(_I), int(r.size)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# -- reference distribution ------------------------------------------------
def gmm_logpdf(x, w, mu, sigma) -> float:
    x, w, mu, sigma = _f64(x), _f64(w), _f64(mu), _f64(sigma)
    return float(lib().orc_gmm_logpdf(_p(x), x.size, w.size, _p(w), _p(mu), _p(sigma)))


def gmm_score(x, w, mu, sigma):
    x, w, mu, sigma = _f64(x), _f64(w), _f64(mu), _f64(sigma)
    T, d = x.shape
    out = np.empty((T, d))
    lib().orc_gmm_score(_p(x), T, d, w.size, _p(w), _p(mu), _p(sigma), _p(out))
    return out


# -- SVGD field (Eq. 4) ----------------------------------------------------
def svgd_field(x, score, h, rows=None):
    x, score = _f64(x), _f64(score)
    T, d = x.shape
    keep, rp, nr = _rows(rows)
    out = np.empty((nr if rows is not None else T, d))
    lib().orc_svgd_field(_p(x), T, d, _p(score), float(h), rp, nr, _p(out))
    return out


def svgd_field_vjp(x, score, h, abar):
    """Gradient of <abar, svgd_field(x, score, h)>: (xbar [T,d] with the score
    held fixed, sbar [T,d] = d/dscore)."""
    x, score, abar = _f64(x), _f64(score), _f64(abar)
    T, d = x.shape
    xbar, sbar = np.empty((T, d)), np.empty((T, d))
    lib().orc_svgd_field_vjp(_p(x), T, d, _p(score), float(h), _p(abar), _p(xbar), _p(sbar))
    return xbar, sbar


def gmm_score_vjp(x, w, mu, sigma, sbar):
    """Reverse mode of gmm_score for cotangents sbar [T,d]: (xbar [T,d] =
    J' sbar per point, wbar [K], mubar [K,d], sigmabar [K])."""
    x, w, mu, sigma, sbar = _f64(x), _f64(w), _f64(mu), _f64(sigma), _f64(sbar)
    T, d = x.shape
    K = w.size
    xbar = np.zeros((T, d))
    wbar, mubar, sbar_s = np.empty(K), np.empty((K, d)), np.empty(K)
    lib().orc_gmm_score_vjp(_p(x), T, d, K, _p(w), _p(mu), _p(sigma), _p(sbar), _p(xbar), _p(wbar), _p(mubar),
                            _p(sbar_s))
    return xbar, wbar, mubar, sbar_s


def svgd_gmm_field_vjp(x, w, mu, sigma, h, abar):
    """Gradient of <abar, svgd_field(x, gmm_score(x), h)> with respect to x
    (through the kernel and the score) and the mixture (w, mu, sigma)."""
    score = gmm_score(x, w, mu, sigma)
    xk, sb = svgd_field_vjp(x, score, h, abar)
    xs, wbar, mubar, sigbar = gmm_score_vjp(x, w, mu, sigma, sb)
    return xk + xs, wbar, mubar, sigbar


# -- Sinkhorn (Eq. 5-7) ----------------------------------------------------
def sinkhorn_g_update(x, y, eps, f, rows=None):
    x, y, f = _f64(x), _f64(y), _f64(f)
    T, d = x.shape
    M = y.shape[0]
    keep, rp, nr = _rows(rows)
    out = np.empty(nr if rows is not None else M)
    lib().orc_sinkhorn_g_update(_p(x), T, _p(y), M, d, float(eps), _p(f), rp, nr, _p(out))
    return out


def sinkhorn_f_update(x, y, b, eps, g, rows=None):
    x, y, g = _f64(x), _f64(y), _f64(g)
    b = None if b is None else _f64(b)
    T, d = x.shape
    M = y.shape[0]
    keep, rp, nr = _rows(rows)
    out = np.empty(nr if rows is not None else T)
    lib().orc_sinkhorn_f_update(_p(x), T, _p(y), M, _p(b), d, float(eps), _p(g), rp, nr, _p(out))
    return out


def sinkhorn_p_update(x, eps, p_old, rows=None):
    x, p_old = _f64(x), _f64(p_old)
    T, d = x.shape
    keep, rp, nr = _rows(rows)
    out = np.empty(nr if rows is not None else T)
    lib().orc_sinkhorn_p_update(_p(x), T, d, float(eps), _p(p_old), rp, nr, _p(out))
    return out


def sinkhorn(x, y, b, eps, n_iter, f=None, g=None, p=None):
    """Fixed-iteration log-domain Sinkhorn; cold start unless f, g, p given."""
    x, y = _f64(x), _f64(y)
    b = None if b is None else _f64(b)
    T, d = x.shape
    M = y.shape[0]
    warm = f is not None
    f = np.zeros(T) if f is None else _f64(f).copy()
    g = np.zeros(M) if g is None else _f64(g).copy()
    p = np.zeros(T) if p is None else _f64(p).copy()
    lib().orc_sinkhorn(_p(x), T, _p(y), M, _p(b), d, float(eps), int(n_iter),
                       int(warm), _p(f), _p(g), _p(p))
    return f, g, p


def anneal_eps(eps, eps_start, eps_decay, t) -> float:
    return float(lib().orc_anneal_eps(float(eps), float(eps_start), float(eps_decay), int(t)))


def sinkhorn_annealed(x, y, b, eps, n_iter, eps_start, eps_decay, f=None, g=None, p=None):
    """Fixed-iteration Sinkhorn with eps_t = max(eps, eps_start eps_decay^t)."""
    x, y = _f64(x), _f64(y)
    b = None if b is None else _f64(b)
    T, d = x.shape
    M = y.shape[0]
    warm = f is not None
    f = np.zeros(T) if f is None else _f64(f).copy()
    g = np.zeros(M) if g is None else _f64(g).copy()
    p = np.zeros(T) if p is None else _f64(p).copy()
    lib().orc_sinkhorn_annealed(_p(x), T, _p(y), M, _p(b), d, float(eps), int(n_iter), float(eps_start),
                                float(eps_decay), int(warm), _p(f), _p(g), _p(p))
    return f, g, p


def density_value(density, x) -> float:
    m = _f64(density)
    xv = _f64(x)
    return float(lib().orc_density_value(_p(m), int(m.shape[0]), int(m.shape[1]), _p(xv)))


def density_score(density, x):
    """grad log q of the bilinear interpolant of the pixel density [H, W] at x [T, 2]."""
    m, xv = _f64(density), _f64(x)
    T = xv.shape[0]
    out = np.empty((T, 2))
    lib().orc_density_score(_p(m), int(m.shape[0]), int(m.shape[1]), _p(xv), T, _p(out))
    return out


def sinkhorn_field(x, y, b, eps, g, p, rows=None):
    x, y, g, p = _f64(x), _f64(y), _f64(g), _f64(p)
    b = None if b is None else _f64(b)
    T, d = x.shape
    M = y.shape[0]
    keep, rp, nr = _rows(rows)
    out = np.empty((nr if rows is not None else T, d))
    lib().orc_sinkhorn_field(_p(x), T, _p(y), M, _p(b), d, float(eps), _p(g), _p(p), rp, nr, _p(out))
    return out


def sinkhorn_converge(x, y, b, eps, tol=1e-12, max_iter=100000):
    x, y = _f64(x), _f64(y)
    b = None if b is None else _f64(b)
    T, d = x.shape
    M = y.shape[0]
    f, g, p = np.zeros(T), np.zeros(M), np.zeros(T)
    it = lib().orc_sinkhorn_converge(_p(x), T, _p(y), M, _p(b), d, float(eps), float(tol),
                                     int(max_iter), _p(f), _p(g), _p(p))
    return f, g, p, int(it)


def sinkhorn_marginals(x, y, b, eps, f, g):
    x, y, f, g = _f64(x), _f64(y), _f64(f), _f64(g)
    b = None if b is None else _f64(b)
    T, d = x.shape
    M = y.shape[0]
    rs, cs = np.empty(T), np.empty(M)
    lib().orc_sinkhorn_marginals(_p(x), T, _p(y), M, _p(b), d, float(eps), _p(f), _p(g), _p(rs), _p(cs))
    return rs, cs


def sinkhorn_divergence(x, y, b, eps, tol=1e-10, max_iter=100000) -> float:
    x, y = _f64(x), _f64(y)
    b = None if b is None else _f64(b)
    T, d = x.shape
    M = y.shape[0]
    return float(lib().orc_sinkhorn_divergence(_p(x), T, _p(y), M, _p(b), d, float(eps),
                                               float(tol), int(max_iter)))


def sinkhorn_divergence_iter(x, y, eps, n_iter) -> float:
    """Debiased Sinkhorn divergence of Eq. 6 as the dual value after n_iter
    cold-start iterations, uniform weights on both sets:
        S = <a, f> + <b, g> - <a, p> - <b, q>
    with f, g, p the potentials of sinkhorn(x, y, None, eps, n_iter) and q the
    self potential of y after n_iter averaged self updates (the p output of
    the same iteration run on y against itself)."""
    f, g, p = sinkhorn(x, y, None, eps, n_iter)
    q = sinkhorn(y, y, None, eps, n_iter)[2]
    return float(np.mean(f) + np.mean(g) - np.mean(p) - np.mean(q))


# -- dynamics, linearisation, rollout (Eq. 3, 8) ---------------------------
def step(model, s, u, dt):
    s, u = _f64(s), _f64(u)
    n, m = MODEL_DIMS[model]
    out = np.empty(n)
    lib().orc_step(int(model), _p(s), _p(u), float(dt), _p(out))
    return out


def linearize(model, s, u, dt):
    s, u = _f64(s), _f64(u)
    n, m = MODEL_DIMS[model]
    T = u.shape[0]
    A, B = np.empty((T, n, n)), np.empty((T, n, m))
    lib().orc_linearize(int(model), _p(s), _p(u), T, float(dt), _p(A), _p(B))
    return A, B


def rollout(model, s0, u, dt):
    s0, u = _f64(s0), _f64(u)
    n, m = MODEL_DIMS[model]
    T = u.shape[0]
    s = np.empty((T + 1, n))
    lib().orc_rollout(int(model), _p(s0), _p(u), T, float(dt), _p(s))
    return s


# -- LQR flow matching (Eq. 9-10) ------------------------------------------
def lqr_track(A, B, Q, R, abar):
    """abar[t-1] is the target at t = 1..T; returns v [T,m], z [T+1,n], P_1."""
    A, B, Q, R, abar = _f64(A), _f64(B), _f64(Q), _f64(R), _f64(abar)
    T, n, m = B.shape
    v, z, P1 = np.empty((T, m)), np.empty((T + 1, n)), np.full((n, n), np.nan)
    lib().orc_lqr_track(_p(A), _p(B), _p(Q), _p(R), _p(abar), T, n, m, _p(v), _p(z), _p(P1))
    return v, z, P1


# -- outer iteration -------------------------------------------------------
def solve(model, dt, s0, u0, field, Q, R, eta, n_outer, *, d=2, y=None, b=None,
          gmm=None, eps=0.0, n_iter=0, h=0.0, warm=False, eps_start=0.0, eps_decay=1.0, density=None):
    """Returns (u, s) after n_outer iterations; u0 [T,m] is not modified.
    warm: Sinkhorn potentials carried across outer iterations; eps_start >
    eps: eps-scaling within each field evaluation; density [H, W]: the Stein
    field's reference as a pixel density (instead of gmm)."""
    dens = None if density is None else _f64(density)
    dh, dw = (0, 0) if dens is None else (int(dens.shape[0]), int(dens.shape[1]))
    n, m = MODEL_DIMS[model]
    u = _f64(u0).copy()
    T = u.shape[0]
    s = np.empty((T + 1, n))
    s0 = _f64(s0)
    Q, R = _f64(Q), _f64(R)
    yv = None if y is None else _f64(y)
    bv = None if b is None else _f64(b)
    M = 0 if y is None else yv.shape[0]
    if gmm is not None:
        gw, gmu, gs = (_f64(v) for v in gmm)
        K = gw.size
    else:
        gw = gmu = gs = None
        K = 0
    rc = lib().orc_solve_ex(int(model), T, float(dt), _p(s0), int(field), int(d), _p(yv), _p(bv), M, K,
                            _p(gw), _p(gmu), _p(gs), float(eps), int(n_iter), float(h), _p(Q), _p(R),
                            float(eta), int(n_outer), _p(u), _p(s), int(warm), float(eps_start),
                            float(eps_decay), _p(dens), dh, dw)
    if rc != 0:
        raise ValueError("orc_solve: bad arguments")
    return u, s


# -- adjoints (reverse mode of the functions above) -------------------------
def sinkhorn_field_vjp(x, y, b, eps, n_iter, abar):
    """Gradient of <abar, field(x, y, b)> after n_iter cold-start iterations.

    Returns (xbar [T,d], ybar [M,d], bbar [M] or None)."""
    x, y, abar = _f64(x), _f64(y), _f64(abar)
    b = None if b is None else _f64(b)
    T, d = x.shape
    M = y.shape[0]
    xbar, ybar = np.zeros((T, d)), np.zeros((M, d))
    bbar = None if b is None else np.zeros(M)
    lib().orc_sinkhorn_field_vjp(_p(x), T, _p(y), M, _p(b), d, float(eps), int(n_iter), _p(abar),
                                 _p(xbar), _p(ybar), _p(bbar))
    return xbar, ybar, bbar


def lqr_vjp(A, B, Q, R, vbar):
    """Gradient of <vbar, v(abar)> with respect to abar (v is linear in abar)."""
    A, B, Q, R, vbar = _f64(A), _f64(B), _f64(Q), _f64(R), _f64(vbar)
    T, n, m = B.shape
    out = np.empty((T, n))
    lib().orc_lqr_vjp(_p(A), _p(B), _p(Q), _p(R), _p(vbar), T, n, m, _p(out))
    return out


def rollout_vjp(model, s, u, dt, sbar):
    """Gradient of <sbar, rollout(s0, u)> at the trajectory s: (ubar, s0bar)."""
    s, u, sbar = _f64(s), _f64(u), _f64(sbar)
    n, m = MODEL_DIMS[model]
    T = u.shape[0]
    ubar, s0bar = np.empty((T, m)), np.zeros(n)
    lib().orc_rollout_vjp(int(model), _p(s), _p(u), T, float(dt), _p(sbar), _p(ubar), _p(s0bar))
    return ubar, s0bar


def solve_sinkhorn_grad(model, dt, s0, u0, d, y, b, eps, n_iter, Q, R, eta, n_outer,
                        y_loss, b_loss, eps_loss):
    """Loss S_eps_loss(trajectory after n_outer iterations, (y_loss, b_loss)) and
    its gradient with respect to (y, b, s0).  Time-invariant models only."""
    n, m = MODEL_DIMS[model]
    s0, u0, y, Q, R, yl = _f64(s0), _f64(u0), _f64(y), _f64(Q), _f64(R), _f64(y_loss)
    b = None if b is None else _f64(b)
    bl = None if b_loss is None else _f64(b_loss)
    T = u0.shape[0]
    M, ML = y.shape[0], yl.shape[0]
    ybar, s0bar = np.zeros((M, d)), np.zeros(n)
    bbar = None if b is None else np.zeros(M)
    L = lib().orc_solve_sinkhorn_grad(int(model), T, float(dt), _p(s0), int(d), _p(y), _p(b), M,
                                      float(eps), int(n_iter), _p(Q), _p(R), float(eta),
                                      int(n_outer), _p(u0), _p(yl), _p(bl), ML, float(eps_loss),
                                      _p(ybar), _p(bbar), _p(s0bar))
    if not np.isfinite(L):
        raise ValueError("orc_solve_sinkhorn_grad: bad arguments")
    return float(L), ybar, bbar, s0bar


def solve_history(model, dt, s0, u0, Q, R, eta, n_outer, *, d, y, b, eps, n_iter):
    """Trajectories s^0..s^K of a Sinkhorn solve: [K+1][T+1][n] (s^k after k updates)."""
    u = _f64(u0).copy()
    hist = [rollout(model, s0, u, dt)]
    for _ in range(n_outer):
        u, s = solve(model, dt, s0, u, FIELD_SINKHORN, Q, R, eta, 1, d=d, y=y, b=b, eps=eps,
                     n_iter=n_iter)
        hist.append(s)
    return np.stack(hist)


def solve_backward(model, dt, d, y, b, eps, n_iter, Q, R, eta, s_hist, sbar_K):
    """Reverse sweep through K = len(s_hist) outer iterations given the
    checkpoints s_hist [K][T+1][n] (s^0..s^{K-1}) and dL/ds^K: returns (ybar [M][d], bbar [M] or None, s0bar [n], u0bar [T][m])."""
    n, m = MODEL_DIMS[model]
    y, Q, R, sh, sb = _f64(y), _f64(Q), _f64(R), _f64(s_hist), _f64(sbar_K)
    b = None if b is None else _f64(b)
    n_outer = sh.shape[0]
    T = sh.shape[1] - 1
    M = y.shape[0]
    ybar, s0bar, u0bar = np.zeros((M, d)), np.zeros(n), np.zeros((T, m))
    bbar = None if b is None else np.zeros(M)
    rc = lib().orc_solve_backward(int(model), T, float(dt), int(d), _p(y), _p(b), M, float(eps),
                                  int(n_iter), _p(Q), _p(R), float(eta), int(n_outer), _p(sh), _p(sb),
                                  _p(ybar), _p(bbar), _p(s0bar), _p(u0bar))
    if rc != 0:
        raise ValueError("orc_solve_backward: bad arguments")
    return ybar, bbar, s0bar, u0bar


def solve_backward_svgd(model, dt, d, gmm, h, Q, R, eta, s_hist, sbar_K):
    """Reverse sweep of a Stein-field solve with the mixture gmm = (w, mu,
    sigma) through K = len(s_hist) outer iterations given the checkpoints
    s_hist [K][T+1][n] and dL/ds^K: returns (wbar [K], mubar [K][d],
    sigmabar [K], s0bar [n], u0bar [T][m])."""
    n, m = MODEL_DIMS[model]
    w, mu, sigma = (_f64(v) for v in gmm)
    Q, R, sh, sb = _f64(Q), _f64(R), _f64(s_hist), _f64(sbar_K)
    n_outer = sh.shape[0]
    T = sh.shape[1] - 1
    K = w.size
    wbar, mubar, sigbar = np.zeros(K), np.zeros((K, d)), np.zeros(K)
    s0bar, u0bar = np.zeros(n), np.zeros((T, m))
    rc = lib().orc_solve_backward_svgd(int(model), T, float(dt), int(d), K, _p(w), _p(mu), _p(sigma), float(h),
                                       _p(Q), _p(R), float(eta), int(n_outer), _p(sh), _p(sb), _p(wbar), _p(mubar),
                                       _p(sigbar), _p(s0bar), _p(u0bar))
    if rc != 0:
        raise ValueError("orc_solve_backward_svgd: bad arguments")
    return wbar, mubar, sigbar, s0bar, u0bar
