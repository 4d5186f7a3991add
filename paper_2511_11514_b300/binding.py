"""ctypes binding of libcov.so (declared in include/cov.h).

Argument marshalling only: every function checks torch tensors (device,
dtype, contiguity, shape), passes their data pointers and the current CUDA
stream to the C-ABI call of the same name, and turns a non-OK status into
``CovError``.  All compute runs in the library's CUDA kernels; there is no
fallback path, and loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcov.so")

COV_OK, COV_ERR_INVALID_ARG, COV_ERR_WORKSPACE, COV_ERR_CUDA, COV_ERR_NONFINITE, COV_ERR_TIMEOUT, \
    COV_ERR_UNSUPPORTED = range(7)
SINGLE_INT, DOUBLE_INT, UNICYCLE = 0, 1, 2
FIELD_SVGD, FIELD_SINKHORN = 0, 1
WARM_START = 1
DEV_NONFINITE, DEV_TIMEOUT, DEV_NOT_SPD = 1, 2, 4
MAX_D, MAX_GMM, MAX_N, MAX_M = 6, 32, 4, 3
OPT_ROWS_PER_THREAD, OPT_THREADS, OPT_CTAS_PER_SM, OPT_USE_GRAPH, OPT_SPIN_LIMIT, OPT_TENSOR_CORES = 1, 2, 3, 4, 5, 6
OPT_BATCH_SHARE = 7
BATCH_SHARE_DEFAULT = 12  # the library's default COV_OPT_BATCH_SHARE
TENSOR_CORES_OFF, TENSOR_CORES_ON, TENSOR_CORES_AUTO = 0, 1, 2
MODEL_DIMS = {SINGLE_INT: (2, 2), DOUBLE_INT: (4, 2), UNICYCLE: (3, 2)}

# Every symbol include/cov.h declares.
EXPORTS = (
    "cov_ctx_create", "cov_ctx_destroy", "cov_ctx_reserve", "cov_workspace_size", "cov_ctx_reserve_for",
    "cov_get_device_status", "cov_status_string", "cov_last_cuda_error", "cov_ctx_set_option",
    "cov_gmm_score", "cov_field_svgd", "cov_field_sinkhorn", "cov_field_sinkhorn_noalloc", "cov_linearize",
    "cov_rollout",
    "cov_lqr_track", "cov_solve", "cov_solve_continue", "cov_solve_batched", "cov_workspace_size_batched",
    "cov_probe_peaks", "cov_workspace_size_vjp", "cov_field_sinkhorn_vjp", "cov_workspace_size_lqr_vjp",
    "cov_lqr_vjp", "cov_rollout_vjp", "cov_solve_checkpointed", "cov_workspace_size_backward",
    "cov_solve_backward", "cov_field_sinkhorn_annealed", "cov_density_score", "cov_autotune_sinkhorn",
    "cov_workspace_size_divergence", "cov_sinkhorn_divergence", "cov_workspace_size_svgd_vjp",
    "cov_field_svgd_vjp", "cov_solve_backward_svgd",
)


class CovError(RuntimeError):
    def __init__(self, status, what, detail=""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}{(' (' + detail + ')') if detail else ''}")


_P = ctypes.c_void_p
_i, _f, _d, _ll, _sz = ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_longlong, ctypes.c_size_t


class cov_gmm(ctypes.Structure):
    _fields_ = [("K", _i), ("d", _i), ("w", _P), ("mu", _P), ("sigma", _P)]


class cov_problem(ctypes.Structure):
    _fields_ = [("model", _i), ("T", _i), ("dt", _d), ("s0", _d * MAX_N), ("field", _i), ("d", _i),
                ("y", _P), ("b", _P), ("M", _i), ("eps", _f), ("n_iter", _i), ("gmm", cov_gmm), ("h", _f),
                ("Q", _d * (MAX_N * MAX_N)), ("R", _d * (MAX_M * MAX_M)), ("eta", _d),
                ("eps_start", _f), ("eps_decay", _f), ("warm", _i), ("density", _P), ("density_h", _i),
                ("density_w", _i)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libcov.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libcov.so not found at {path}: run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    sig = {
        "cov_ctx_create": (_i, [ctypes.POINTER(_P), _i, _sz]),
        "cov_ctx_destroy": (None, [_P]),
        "cov_ctx_reserve": (_i, [_P, _sz]),
        "cov_workspace_size": (_sz, [_i, _i, _i, _i, _i]),
        "cov_ctx_reserve_for": (_i, [_P, _i, _i, _i, _i, _i]),
        "cov_get_device_status": (_i, [_P, _P, ctypes.POINTER(_i)]),
        "cov_status_string": (ctypes.c_char_p, [_i]),
        "cov_last_cuda_error": (ctypes.c_char_p, [_P]),
        "cov_ctx_set_option": (_i, [_P, _i, _ll]),
        "cov_gmm_score": (_i, [_P, _P, _i, _i, ctypes.POINTER(cov_gmm), _P, _P]),
        "cov_field_svgd": (_i, [_P, _P, _i, _i, _P, ctypes.POINTER(cov_gmm), _f, _P, _P]),
        "cov_field_sinkhorn": (_i, [_P, _P, _i, _P, _P, _i, _i, _f, _i, _i, _P, _P, _P, _P, _P]),
        "cov_field_sinkhorn_noalloc": (_i, [_P, _i, _P, _P, _i, _i, _f, _i, _i, _P, _P, _P, _P, _P]),
        "cov_linearize": (_i, [_P, _i, _P, _P, _i, _d, _P, _P, _P]),
        "cov_rollout": (_i, [_P, _i, _P, _P, _i, _d, _P, _P]),
        "cov_lqr_track": (_i, [_P, _P, _P, _P, _P, _P, _i, _i, _i, _P, _P, _P]),
        "cov_solve": (_i, [_P, ctypes.POINTER(cov_problem), _i, _P, _P, _P]),
        "cov_solve_continue": (_i, [_P, ctypes.POINTER(cov_problem), _i, _P, _P, _P]),
        "cov_solve_batched": (_i, [_P, ctypes.POINTER(cov_problem), _i, _i, ctypes.POINTER(_P),
                                   ctypes.POINTER(_P), _P]),
        "cov_workspace_size_batched": (_sz, [ctypes.POINTER(cov_problem), _i]),
        "cov_probe_peaks": (_i, [_P, _i, ctypes.POINTER(_d), _P]),
        "cov_density_score": (_i, [_P, _P, _i, _i, _P, _i, _P, _P]),
        "cov_autotune_sinkhorn": (_i, [_P, _P, _i, _P, _P, _i, _i, _f, ctypes.POINTER(_i), ctypes.POINTER(_i),
                                       ctypes.POINTER(_d), _P]),
        "cov_field_sinkhorn_annealed": (_i, [_P, _P, _i, _P, _P, _i, _i, _f, _i, _f, _f, _i, _P, _P, _P, _P, _P]),
        "cov_workspace_size_vjp": (_sz, [_i, _i, _i, _i]),
        "cov_field_sinkhorn_vjp": (_i, [_P, _P, _i, _P, _P, _i, _i, _f, _i, _P, _P, _P, _P, _P]),
        "cov_workspace_size_lqr_vjp": (_sz, [_i, _i, _i]),
        "cov_lqr_vjp": (_i, [_P, _P, _P, _P, _P, _P, _i, _i, _i, _P, _P]),
        "cov_rollout_vjp": (_i, [_P, _i, _P, _P, _i, _d, _P, _P, _P, _P]),
        "cov_solve_checkpointed": (_i, [_P, ctypes.POINTER(cov_problem), _i, _P, _P, _P, _i, _P]),
        "cov_workspace_size_backward": (_sz, [ctypes.POINTER(cov_problem), _i, _i]),
        "cov_solve_backward": (_i, [_P, ctypes.POINTER(cov_problem), _i, _P, _P, _P, _P, _P, _P, _P, _P]),
        "cov_workspace_size_divergence": (_sz, [_i, _i, _i]),
        "cov_sinkhorn_divergence": (_i, [_P, _P, _i, _P, _P, _i, _i, _f, _i, _P, _i, _P, _P, _P]),
        "cov_workspace_size_svgd_vjp": (_sz, [_i, _i, _i]),
        "cov_solve_backward_svgd": (_i, [_P, ctypes.POINTER(cov_problem), _i, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
        "cov_field_svgd_vjp": (_i, [_P, _P, _i, _i, _P, ctypes.POINTER(cov_gmm), _f, _P, _P, _P, _P, _P, _P,
                                    _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_string(s: int) -> str:
    try:
        return load().cov_status_string(int(s)).decode()
    except Exception:
        return f"status {s}"


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, dtype, shape=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """A libcov context on one CUDA device (owns the workspace)."""

    def __init__(self, device: int | None = None, workspace_bytes: int = 0):
        L = load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        st = L.cov_ctx_create(ctypes.byref(h), self.device, int(workspace_bytes))
        if st != COV_OK:
            raise CovError(st, "cov_ctx_create")
        self.h = h
        self._keep = []
        self._options = {}      # options set through set_option (the tuner's cache keys read them)
        self._cache = {}        # persistent buffers of the graph-friendly gradient calls
        self._grad_token = 0    # identifies the latest recording forward of grad_forward

    def close(self):
        if getattr(self, "h", None):
            load().cov_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st, what):
        if st != COV_OK:
            detail = load().cov_last_cuda_error(self.h).decode() if st == COV_ERR_CUDA else ""
            raise CovError(st, what, detail)

    def reserve_for(self, T, M=0, d=2, n=0, m=0):
        self._check(load().cov_ctx_reserve_for(self.h, int(T), int(M), int(d), int(n), int(m)), "cov_ctx_reserve_for")

    def reserve(self, nbytes: int):
        if int(nbytes) <= 0:
            raise CovError(COV_ERR_INVALID_ARG, "workspace size")
        self._check(load().cov_ctx_reserve(self.h, int(nbytes)), "cov_ctx_reserve")

    def set_option(self, key: int, value: int):
        self._check(load().cov_ctx_set_option(self.h, int(key), int(value)), "cov_ctx_set_option")
        self._options[int(key)] = int(value)

    def option(self, key: int, default: int):
        """The value last set for `key` through set_option, else `default`."""
        return self._options.get(int(key), default)

    def device_status(self, stream=None):
        """(status code, COV_DEV_* bits); synchronises the stream, clears the bits."""
        fl = ctypes.c_int(0)
        st = load().cov_get_device_status(self.h, _stream(stream), ctypes.byref(fl))
        return st, fl.value


def workspace_size(T, M=0, d=2, n=0, m=0) -> int:
    return int(load().cov_workspace_size(int(T), int(M), int(d), int(n), int(m)))


def _gmm_struct(gmm, d):
    """(struct, keep-alive arrays) for gmm = (w, mu, sigma) host arrays."""
    w, mu, sigma = (np.ascontiguousarray(np.asarray(v, dtype=np.float32)) for v in gmm)
    g = cov_gmm(K=int(w.size), d=int(d), w=w.ctypes.data_as(_P), mu=mu.ctypes.data_as(_P),
                sigma=sigma.ctypes.data_as(_P))
    return g, (w, mu, sigma)


def cov_autotune_sinkhorn(ctx: Context, x, y, eps, b=None, stream=None):
    """Sweep the tile shapes on these inputs (C side), apply the fastest;
    returns (R, ctas_per_sm, [(R, cap, us per iteration), ...])."""
    T, d = x.shape
    M = y.shape[0]
    ctx.reserve_for(T, M, d)
    bR, bC = ctypes.c_int(0), ctypes.c_int(0)
    sw = (ctypes.c_double * 18)()
    st = load().cov_autotune_sinkhorn(ctx.h, _ptr(x, torch.float32, name="x"), T, _ptr(y, torch.float32, (M, d), "y"),
                                      _ptr(b, torch.float32, (M,), "b"), M, d, float(eps), ctypes.byref(bR),
                                      ctypes.byref(bC), sw, _stream(stream))
    ctx._check(st, "cov_autotune_sinkhorn")
    rows = [(int(sw[3 * k]), int(sw[3 * k + 1]), float(sw[3 * k + 2])) for k in range(6)]
    return bR.value, bC.value, rows


def cov_density_score(ctx: Context, density, x, out=None, stream=None):
    """grad log q of the bilinear interpolant of the pixel density [H, W] at x [T, 2]."""
    T = x.shape[0]
    H, W = density.shape
    out = torch.empty((T, 2), device=x.device, dtype=torch.float32) if out is None else out
    st = load().cov_density_score(ctx.h, _ptr(density, torch.float32, name="density"), int(H), int(W),
                                  _ptr(x, torch.float32, (T, 2), "x"), T, _ptr(out, torch.float32, (T, 2), "out"),
                                  _stream(stream))
    ctx._check(st, "cov_density_score")
    return out


def cov_gmm_score(ctx: Context, x, gmm, out=None, stream=None):
    T, d = x.shape
    out = torch.empty_like(x) if out is None else out
    g, keep = _gmm_struct(gmm, d)
    st = load().cov_gmm_score(ctx.h, _ptr(x, torch.float32, name="x"), T, d, ctypes.byref(g),
                              _ptr(out, torch.float32, (T, d), "out"), _stream(stream))
    ctx._check(st, "cov_gmm_score")
    return out


def cov_field_svgd(ctx: Context, x, h, score=None, gmm=None, out=None, stream=None):
    """Stein variational field (Eq. 4) at all rows of x [T, d]."""
    T, d = x.shape
    ctx.reserve_for(T, 0, d)
    out = torch.empty_like(x) if out is None else out
    g = None
    keep = None
    if score is None:
        if gmm is None:
            raise ValueError("need score or gmm")
        g, keep = _gmm_struct(gmm, d)
    st = load().cov_field_svgd(ctx.h, _ptr(x, torch.float32, name="x"), T, d,
                               _ptr(score, torch.float32, (T, d), "score"),
                               ctypes.byref(g) if g is not None else None, float(h),
                               _ptr(out, torch.float32, (T, d), "out"), _stream(stream))
    ctx._check(st, "cov_field_svgd")
    return out


def cov_field_svgd_vjp(ctx: Context, x, h, abar, score=None, gmm=None, want_sbar=True, want_gmm=True,
                       stream=None):
    """Reverse mode of the Stein field (Eq. 4) for L = <abar, field>.  With
    a score tensor: (xbar, sbar) with the score held fixed.  With gmm = (w,
    mu, sigma): (xbar, sbar, (wbar, mubar, sigmabar)), xbar the total
    gradient through the kernel and the mixture score."""
    T, d = x.shape
    K = 0 if score is not None else len(gmm[0])
    need = int(load().cov_workspace_size_svgd_vjp(T, d, K))
    if need == 0:
        raise CovError(COV_ERR_INVALID_ARG, "cov_workspace_size_svgd_vjp")
    ctx._check(load().cov_ctx_reserve(ctx.h, need), "cov_ctx_reserve")
    dev = x.device
    xbar = torch.empty_like(x)
    sbar = torch.empty_like(x) if want_sbar else None
    g = arrs = None
    wb = mb = sb = None
    if score is None:
        g, arrs = _gmm_struct(gmm, d)
        if want_gmm:
            wb = torch.empty(K, device=dev, dtype=torch.float32)
            mb = torch.empty((K, d), device=dev, dtype=torch.float32)
            sb = torch.empty(K, device=dev, dtype=torch.float32)
    st = load().cov_field_svgd_vjp(
        ctx.h, _ptr(x, torch.float32, name="x"), T, d,
        _ptr(score, torch.float32, (T, d), "score") if score is not None else None,
        ctypes.byref(g) if g is not None else None, float(h), _ptr(abar, torch.float32, (T, d), "abar"),
        _ptr(xbar, torch.float32, (T, d), "xbar"), _ptr(sbar, torch.float32, (T, d), "sbar") if want_sbar else None,
        _ptr(wb, torch.float32, (K,), "wbar") if wb is not None else None,
        _ptr(mb, torch.float32, (K, d), "mubar") if mb is not None else None,
        _ptr(sb, torch.float32, (K,), "sigmabar") if sb is not None else None, _stream(stream))
    ctx._check(st, "cov_field_svgd_vjp")
    del arrs
    if score is not None:
        return xbar, sbar
    return xbar, sbar, (wb, mb, sb)


def cov_field_sinkhorn(ctx: Context, x, y, eps, n_iter, b=None, f=None, g=None, p=None, warm=False,
                       field=True, out=None, stream=None):
    """Sinkhorn-divergence field (Eq. 5-7).  Returns (a, f, g, p); f, g, p
    are allocated when not given.  a is None when field=False."""
    T, d = x.shape
    M = y.shape[0]
    ctx.reserve_for(T, M, d)
    dev = x.device
    f = torch.empty(T, device=dev, dtype=torch.float32) if f is None else f
    g = torch.empty(M, device=dev, dtype=torch.float32) if g is None else g
    p = torch.empty(T, device=dev, dtype=torch.float32) if p is None else p
    if field and out is None:
        out = torch.empty_like(x)
    st = load().cov_field_sinkhorn(
        ctx.h, _ptr(x, torch.float32, name="x"), T, _ptr(y, torch.float32, (M, d), "y"),
        _ptr(b, torch.float32, (M,), "b"), M, d, float(eps), int(n_iter), WARM_START if warm else 0,
        _ptr(f, torch.float32, (T,), "f"), _ptr(g, torch.float32, (M,), "g"), _ptr(p, torch.float32, (T,), "p"),
        _ptr(out, torch.float32, (T, d), "out") if field else None, _stream(stream))
    ctx._check(st, "cov_field_sinkhorn")
    return (out if field else None), f, g, p


def cov_sinkhorn_divergence(ctx: Context, x, y, eps, n_iter, b=None, q_ref=None, q_given=False, grad=True,
                            stream=None):
    """Debiased Sinkhorn divergence of Eq. 6 after n_iter iterations (dual
    value) and its gradient -(1/T) field with respect to x.  Returns
    (value: 0-dim float64 CUDA tensor, grad [T, d] or None, q_ref [M]): q_ref
    is the reference's self potential, computed here unless q_given (then
    the given tensor is read; pass the q_ref of an earlier call on the same
    y, eps, n_iter)."""
    T, d = x.shape
    M = y.shape[0]
    need = int(load().cov_workspace_size_divergence(T, M, d))
    if need == 0:
        raise CovError(COV_ERR_INVALID_ARG, "cov_workspace_size_divergence")
    ctx._check(load().cov_ctx_reserve(ctx.h, need), "cov_ctx_reserve")
    dev = x.device
    if q_ref is None:
        if q_given:
            raise CovError(COV_ERR_INVALID_ARG, "cov_sinkhorn_divergence", "q_given without q_ref")
        q_ref = torch.empty(M, device=dev, dtype=torch.float32)
    value = torch.empty((), device=dev, dtype=torch.float64)
    g_out = torch.empty_like(x) if grad else None
    st = load().cov_sinkhorn_divergence(
        ctx.h, _ptr(x, torch.float32, name="x"), T, _ptr(y, torch.float32, (M, d), "y"),
        _ptr(b, torch.float32, (M,), "b"), M, d, float(eps), int(n_iter), _ptr(q_ref, torch.float32, (M,), "q_ref"),
        1 if q_given else 0, _ptr(value, torch.float64, (), "value"),
        _ptr(g_out, torch.float32, (T, d), "grad") if grad else None, _stream(stream))
    ctx._check(st, "cov_sinkhorn_divergence")
    return value, g_out, q_ref


def cov_field_sinkhorn_annealed(ctx: Context, x, y, eps, n_iter, eps_start, eps_decay, b=None, f=None, g=None,
                                p=None, warm=False, field=True, out=None, stream=None):
    """cov_field_sinkhorn with eps-scaling: iteration t at max(eps, eps_start eps_decay^t)."""
    T, d = x.shape
    M = y.shape[0]
    ctx.reserve_for(T, M, d)
    dev = x.device
    f = torch.empty(T, device=dev, dtype=torch.float32) if f is None else f
    g = torch.empty(M, device=dev, dtype=torch.float32) if g is None else g
    p = torch.empty(T, device=dev, dtype=torch.float32) if p is None else p
    if field and out is None:
        out = torch.empty_like(x)
    st = load().cov_field_sinkhorn_annealed(
        ctx.h, _ptr(x, torch.float32, name="x"), T, _ptr(y, torch.float32, (M, d), "y"),
        _ptr(b, torch.float32, (M,), "b"), M, d, float(eps), int(n_iter), float(eps_start), float(eps_decay),
        WARM_START if warm else 0, _ptr(f, torch.float32, (T,), "f"), _ptr(g, torch.float32, (M,), "g"),
        _ptr(p, torch.float32, (T,), "p"), _ptr(out, torch.float32, (T, d), "out") if field else None,
        _stream(stream))
    ctx._check(st, "cov_field_sinkhorn_annealed")
    return (out if field else None), f, g, p


def cov_linearize(ctx: Context, model, s, u, dt, A=None, B=None, stream=None):
    n, m = MODEL_DIMS[model]
    T = u.shape[0]
    A = torch.empty((T, n, n), device=u.device, dtype=torch.float64) if A is None else A
    B = torch.empty((T, n, m), device=u.device, dtype=torch.float64) if B is None else B
    st = load().cov_linearize(ctx.h, int(model), _ptr(s, torch.float64, (T + 1, n), "s"),
                              _ptr(u, torch.float64, (T, m), "u"), T, float(dt),
                              _ptr(A, torch.float64, (T, n, n), "A"), _ptr(B, torch.float64, (T, n, m), "B"),
                              _stream(stream))
    ctx._check(st, "cov_linearize")
    return A, B


def cov_rollout(ctx: Context, model, s0, u, dt, out=None, stream=None):
    n, m = MODEL_DIMS[model]
    T = u.shape[0]
    ctx.reserve_for(T, 0, 1, n, m)
    s0h = np.ascontiguousarray(np.asarray(s0, dtype=np.float64))
    out = torch.empty((T + 1, n), device=u.device, dtype=torch.float64) if out is None else out
    st = load().cov_rollout(ctx.h, int(model), s0h.ctypes.data_as(_P), _ptr(u, torch.float64, (T, m), "u"), T,
                            float(dt), _ptr(out, torch.float64, (T + 1, n), "s"), _stream(stream))
    ctx._check(st, "cov_rollout")
    return out


def cov_lqr_track(ctx: Context, A, B, Q, R, abar, want_z=True, stream=None):
    """LQR tracking (Eq. 9-10).  Q [n,n], R [m,m] host arrays; returns (v, z)."""
    T, n, m = B.shape
    ctx.reserve_for(T, 0, 1, n, m)
    Qh = np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
    Rh = np.ascontiguousarray(np.asarray(R, dtype=np.float64))
    if Qh.shape != (n, n) or Rh.shape != (m, m):
        raise ValueError("Q must be [n,n] and R [m,m]")
    v = torch.empty((T, m), device=B.device, dtype=torch.float64)
    z = torch.empty((T + 1, n), device=B.device, dtype=torch.float64) if want_z else None
    st = load().cov_lqr_track(ctx.h, _ptr(A, torch.float64, (T, n, n), "A"), _ptr(B, torch.float64, (T, n, m), "B"),
                              Qh.ctypes.data_as(_P), Rh.ctypes.data_as(_P), _ptr(abar, torch.float64, (T, n), "abar"),
                              T, n, m, _ptr(v, torch.float64, (T, m), "v"),
                              _ptr(z, torch.float64, (T + 1, n), "z") if want_z else None, _stream(stream))
    ctx._check(st, "cov_lqr_track")
    return v, z


def make_problem(model, T, dt, s0, field, Q, R, eta, *, d=2, y=None, b=None, eps=0.0, n_iter=0, gmm=None, h=0.0,
                 eps_start=0.0, eps_decay=1.0, warm=False, density=None):
    """Build a cov_problem; returns (struct, keep-alive list).  eps_start >
    eps turns on eps-scaling; warm carries the Sinkhorn potentials between
    outer iterations."""
    n, m = MODEL_DIMS[model]
    P = cov_problem()
    P.model, P.T, P.dt, P.field, P.d = int(model), int(T), float(dt), int(field), int(d)
    for r in range(n):
        P.s0[r] = float(s0[r])
    Q = np.asarray(Q, dtype=np.float64).reshape(n, n)
    R = np.asarray(R, dtype=np.float64).reshape(m, m)
    for e in range(n * n):
        P.Q[e] = float(Q.flat[e])
    for e in range(m * m):
        P.R[e] = float(R.flat[e])
    P.eta = float(eta)
    P.eps_start, P.eps_decay, P.warm = float(eps_start), float(eps_decay), int(bool(warm))
    keep = []
    if y is not None:
        P.y = _ptr(y, torch.float32, name="y").value
        P.M = int(y.shape[0])
        if b is not None:
            P.b = _ptr(b, torch.float32, (P.M,), "b").value
        P.eps, P.n_iter = float(eps), int(n_iter)
        keep += [y, b]
    if gmm is not None:
        g, arrs = _gmm_struct(gmm, d)
        P.gmm = g
        keep.append(arrs)
        P.h = float(h)
    if density is not None:
        P.density = _ptr(density, torch.float32, name="density").value
        P.density_h, P.density_w = int(density.shape[0]), int(density.shape[1])
        P.h = float(h)
        keep.append(density)
    return P, keep


def cov_solve(ctx: Context, problem, n_outer, u, s_out=None, stream=None):
    """Run n_outer outer iterations in place on u [T, m] (float64); returns s [T+1, n]."""
    P, keep = problem
    n, m = MODEL_DIMS[P.model]
    T = P.T
    ctx.reserve_for(T, P.M, P.d, n, m)
    s_out = torch.empty((T + 1, n), device=u.device, dtype=torch.float64) if s_out is None else s_out
    st = load().cov_solve(ctx.h, ctypes.byref(P), int(n_outer), _ptr(u, torch.float64, (T, m), "u"),
                          _ptr(s_out, torch.float64, (T + 1, n), "s_out"), _stream(stream))
    ctx._check(st, "cov_solve")
    return s_out


def cov_solve_continue(ctx: Context, problem, n_outer, u, s, stream=None):
    """Continue n_outer outer iterations from (u, s), s = rollout of u."""
    P, keep = problem
    n, m = MODEL_DIMS[P.model]
    T = P.T
    ctx.reserve_for(T, P.M, P.d, n, m)
    st = load().cov_solve_continue(ctx.h, ctypes.byref(P), int(n_outer), _ptr(u, torch.float64, (T, m), "u"),
                                   _ptr(s, torch.float64, (T + 1, n), "s"), _stream(stream))
    ctx._check(st, "cov_solve_continue")
    return s


def cov_solve_batched(ctx: Context, problems, n_outer, us, ss=None, stream=None):
    """n_outer outer iterations of independent problems [(struct, keep), ...]
    in one CUDA graph per iteration; us[p] (float64 [T_p, m_p]) are updated in
    place; returns the trajectories ss[p] ([T_p+1, n_p])."""
    n = len(problems)
    arr = (cov_problem * n)(*[pr[0] for pr in problems])
    if ss is None:
        ss = [torch.empty((pr[0].T + 1, MODEL_DIMS[pr[0].model][0]), device=u.device, dtype=torch.float64)
              for pr, u in zip(problems, us)]
    up = (_P * n)(*[_ptr(u, torch.float64, (pr[0].T, MODEL_DIMS[pr[0].model][1]), "u").value
                    for pr, u in zip(problems, us)])
    sp = (_P * n)(*[_ptr(s, torch.float64, (pr[0].T + 1, MODEL_DIMS[pr[0].model][0]), "s").value
                    for pr, s in zip(problems, ss)])
    need = int(load().cov_workspace_size_batched(arr, n))
    if need == 0:
        raise CovError(COV_ERR_INVALID_ARG, "cov_workspace_size_batched")
    ctx._check(load().cov_ctx_reserve(ctx.h, need), "cov_ctx_reserve")
    st = load().cov_solve_batched(ctx.h, arr, n, int(n_outer), up, sp, _stream(stream))
    ctx._check(st, "cov_solve_batched")
    return ss


def cov_probe_peaks(ctx: Context, iters=4096, stream=None):
    out = (ctypes.c_double * 8)()
    st = load().cov_probe_peaks(ctx.h, int(iters), out, _stream(stream))
    ctx._check(st, "cov_probe_peaks")
    keys = ("ffma_lane_ops_s", "ffma2_lane_ops_s", "ex2_lane_ops_s", "dfma_lane_ops_s", "dfma_latency_cycles",
            "sm_clock_mhz", "exp2_fma_values_s", "exp2_fma_max_rel_err")
    return dict(zip(keys, list(out)))


# -- adjoints -------------------------------------------------------------------
def cov_field_sinkhorn_vjp(ctx: Context, x, y, eps, n_iter, abar, b=None, stream=None):
    """(xbar, ybar, bbar) = gradients of <abar, field(x, y, b)> (bbar None for uniform weights)."""
    T, d = x.shape
    M = y.shape[0]
    ctx.reserve(load().cov_workspace_size_vjp(T, M, d, int(n_iter)))
    xbar = torch.empty_like(x)
    ybar = torch.empty_like(y)
    bbar = torch.empty_like(b) if b is not None else None
    st = load().cov_field_sinkhorn_vjp(
        ctx.h, _ptr(x, torch.float32, name="x"), T, _ptr(y, torch.float32, (M, d), "y"),
        _ptr(b, torch.float32, (M,), "b"), M, d, float(eps), int(n_iter), _ptr(abar, torch.float32, (T, d), "abar"),
        _ptr(xbar, torch.float32, (T, d), "xbar"), _ptr(ybar, torch.float32, (M, d), "ybar"),
        _ptr(bbar, torch.float32, (M,), "bbar"), _stream(stream))
    ctx._check(st, "cov_field_sinkhorn_vjp")
    return xbar, ybar, bbar


def cov_lqr_vjp(ctx: Context, A, B, Q, R, vbar, stream=None):
    """abar_bar [T, n]: gradient of <vbar, v(abar)> of cov_lqr_track."""
    T, n, m = B.shape
    ctx.reserve(load().cov_workspace_size_lqr_vjp(T, n, m))
    Qh = np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
    Rh = np.ascontiguousarray(np.asarray(R, dtype=np.float64))
    if Qh.shape != (n, n) or Rh.shape != (m, m):
        raise ValueError("Q must be [n,n] and R [m,m]")
    out = torch.empty((T, n), device=B.device, dtype=torch.float64)
    st = load().cov_lqr_vjp(ctx.h, _ptr(A, torch.float64, (T, n, n), "A"), _ptr(B, torch.float64, (T, n, m), "B"),
                            Qh.ctypes.data_as(_P), Rh.ctypes.data_as(_P), _ptr(vbar, torch.float64, (T, m), "vbar"),
                            T, n, m, _ptr(out, torch.float64, (T, n), "abar_bar"), _stream(stream))
    ctx._check(st, "cov_lqr_vjp")
    return out


def cov_rollout_vjp(ctx: Context, model, s, u, dt, sbar, stream=None):
    """(ubar [T, m], s0bar [n]): gradient of <sbar, rollout(s0, u)> at the trajectory s."""
    n, m = MODEL_DIMS[model]
    T = u.shape[0]
    ctx.reserve(load().cov_workspace_size_lqr_vjp(T, n, m))
    ubar = torch.empty((T, m), device=u.device, dtype=torch.float64)
    s0bar = torch.empty(n, device=u.device, dtype=torch.float64)
    st = load().cov_rollout_vjp(ctx.h, int(model), _ptr(s, torch.float64, (T + 1, n), "s"),
                                _ptr(u, torch.float64, (T, m), "u"), T, float(dt),
                                _ptr(sbar, torch.float64, (T + 1, n), "sbar"), _ptr(ubar, torch.float64, (T, m), "ubar"),
                                _ptr(s0bar, torch.float64, (n,), "s0bar"), _stream(stream))
    ctx._check(st, "cov_rollout_vjp")
    return ubar, s0bar


CKPT_RECORD = 1
BACKWARD_CHECKPOINTS, BACKWARD_REPLAY, BACKWARD_RECORDED = 0, 1, 2


def cov_solve_checkpointed(ctx: Context, problem, n_outer, u, s_out=None, s_hist=None, record=False, stream=None):
    """cov_solve that also returns the checkpoints s_hist [n_outer, T+1, n];
    record=True also keeps every outer iteration's Sinkhorn record for
    cov_solve_backward."""
    P, keep = problem
    n, m = MODEL_DIMS[P.model]
    T = P.T
    ctx.reserve_for(T, P.M, P.d, n, m)
    if record:
        need = int(load().cov_workspace_size_backward(ctypes.byref(P), int(n_outer), BACKWARD_RECORDED))
        if need == 0:
            raise CovError(COV_ERR_UNSUPPORTED, "recording solve (Sinkhorn field, time-invariant model, d <= 3)")
        ctx.reserve(need)
    s_out = torch.empty((T + 1, n), device=u.device, dtype=torch.float64) if s_out is None else s_out
    if s_hist is None:
        s_hist = torch.empty((max(int(n_outer), 1), T + 1, n), device=u.device, dtype=torch.float64)
    st = load().cov_solve_checkpointed(ctx.h, ctypes.byref(P), int(n_outer), _ptr(u, torch.float64, (T, m), "u"),
                                       _ptr(s_out, torch.float64, (T + 1, n), "s_out"),
                                       _ptr(s_hist, torch.float64, name="s_hist"), CKPT_RECORD if record else 0,
                                       _stream(stream))
    ctx._check(st, "cov_solve_checkpointed")
    return s_out, s_hist


def cov_solve_backward(ctx: Context, problem, n_outer, u0, sbar_K, s_hist=None, stream=None):
    """(ybar [M, d], bbar [M] or None, s0bar [n], u0bar [T, m]) = dL/d(y, b, s0, u0)
    given dL/ds^K = sbar_K and the checkpoints (replayed from u0 when None)."""
    P, keep = problem
    n, m = MODEL_DIMS[P.model]
    T = P.T
    mode = BACKWARD_REPLAY if s_hist is None else BACKWARD_CHECKPOINTS
    need = int(load().cov_workspace_size_backward(ctypes.byref(P), int(n_outer), mode))
    if need == 0:
        raise CovError(COV_ERR_UNSUPPORTED, "cov_solve_backward (Sinkhorn field, time-invariant model, d <= 3)")
    ctx.reserve(need)  # never shrinks: a recording forward's workspace (larger) is kept
    dev = u0.device
    ybar = torch.empty((P.M, P.d), device=dev, dtype=torch.float32)
    bbar = torch.empty(P.M, device=dev, dtype=torch.float32) if P.b else None
    s0bar = torch.empty(n, device=dev, dtype=torch.float64)
    u0bar = torch.empty((T, m), device=dev, dtype=torch.float64)
    hist_p = None
    if s_hist is not None:
        hist_p = _ptr(s_hist, torch.float64, name="s_hist")
        if s_hist.shape[0] < int(n_outer) or tuple(s_hist.shape[1:]) != (T + 1, n):
            raise ValueError("s_hist must be [n_outer, T+1, n]")
    st = load().cov_solve_backward(ctx.h, ctypes.byref(P), int(n_outer), _ptr(u0, torch.float64, (T, m), "u0"),
                                   hist_p, _ptr(sbar_K, torch.float64, (T + 1, n), "sbar_K"),
                                   _ptr(ybar, torch.float32, (P.M, P.d), "ybar"),
                                   _ptr(bbar, torch.float32, (P.M,), "bbar"), _ptr(s0bar, torch.float64, (n,), "s0bar"),
                                   _ptr(u0bar, torch.float64, (T, m), "u0bar"), _stream(stream))
    ctx._check(st, "cov_solve_backward")
    return ybar, bbar, s0bar, u0bar


def cov_solve_backward_svgd(ctx: Context, problem, n_outer, u0, sbar_K, s_hist=None, stream=None):
    """(wbar [K], mubar [K, d], sigmabar [K], s0bar [n], u0bar [T, m]) = dL/d(mixture
    weights, means, standard deviations, s0, u0) of a Stein-field solve with a
    mixture reference, given dL/ds^K = sbar_K and the checkpoints (replayed
    from u0 when None)."""
    P, keep = problem
    n, m = MODEL_DIMS[P.model]
    T, K, d = P.T, P.gmm.K, P.d
    mode = BACKWARD_REPLAY if s_hist is None else BACKWARD_CHECKPOINTS
    need = int(load().cov_workspace_size_backward(ctypes.byref(P), int(n_outer), mode))
    if need == 0:
        raise CovError(COV_ERR_UNSUPPORTED, "cov_solve_backward_svgd (Stein field, mixture, time-invariant model)")
    ctx.reserve(need)
    dev = u0.device
    wbar = torch.empty(K, device=dev, dtype=torch.float32)
    mubar = torch.empty((K, d), device=dev, dtype=torch.float32)
    sigmabar = torch.empty(K, device=dev, dtype=torch.float32)
    s0bar = torch.empty(n, device=dev, dtype=torch.float64)
    u0bar = torch.empty((T, m), device=dev, dtype=torch.float64)
    hist_p = None
    if s_hist is not None:
        hist_p = _ptr(s_hist, torch.float64, name="s_hist")
        if s_hist.shape[0] < int(n_outer) or tuple(s_hist.shape[1:]) != (T + 1, n):
            raise ValueError("s_hist must be [n_outer, T+1, n]")
    st = load().cov_solve_backward_svgd(ctx.h, ctypes.byref(P), int(n_outer), _ptr(u0, torch.float64, (T, m), "u0"),
                                        hist_p, _ptr(sbar_K, torch.float64, (T + 1, n), "sbar_K"),
                                        _ptr(wbar, torch.float32, (K,), "wbar"),
                                        _ptr(mubar, torch.float32, (K, d), "mubar"),
                                        _ptr(sigmabar, torch.float32, (K,), "sigmabar"),
                                        _ptr(s0bar, torch.float64, (n,), "s0bar"),
                                        _ptr(u0bar, torch.float64, (T, m), "u0bar"), _stream(stream))
    ctx._check(st, "cov_solve_backward_svgd")
    return wbar, mubar, sigmabar, s0bar, u0bar


# -- graph-friendly forward/backward pair (used by autograd) -------------------
# cov_solve_checkpointed and cov_solve_backward replay a cached CUDA graph when
# called again with the same problem, sizes and pointers.  These two helpers
# keep their device buffers in the context (copying inputs in and results
# out), so repeated training steps hit the cached graphs.
def _cached(ctx: Context, name, shape, dtype, device):
    key = (name, tuple(int(v) for v in shape), dtype, str(device))
    t = ctx._cache.get(key)
    if t is None:
        t = torch.empty(tuple(shape), dtype=dtype, device=device)
        ctx._cache[key] = t
    return t


def grad_forward(ctx: Context, problem, n_outer, u0, y, b=None, stream=None):
    """Recording forward from u0 (not modified) on the reference (y, b):
    returns (s_K, s_hist, token, problem'), s_K and s_hist fresh tensors;
    token names this forward and problem' (the problem on the context's copies
    of y and b) is what grad_backward takes."""
    P0, keep = problem
    n, m = MODEL_DIMS[P0.model]
    T = P0.T
    dev = u0.device
    yc = _cached(ctx, "y", tuple(y.shape), torch.float32, dev)
    yc.copy_(y)
    P = cov_problem.from_buffer_copy(P0)
    P.y = _ptr(yc, torch.float32, name="y").value
    if b is not None:
        bc = _cached(ctx, "b", tuple(b.shape), torch.float32, dev)
        bc.copy_(b)
        P.b = _ptr(bc, torch.float32, name="b").value
    else:
        P.b = None
    pr = (P, keep)
    u = _cached(ctx, "u", (T, m), torch.float64, dev)
    s_out = _cached(ctx, "s_out", (T + 1, n), torch.float64, dev)
    hist = _cached(ctx, "hist", (max(int(n_outer), 1), T + 1, n), torch.float64, dev)
    u.copy_(u0)
    cov_solve_checkpointed(ctx, pr, n_outer, u, s_out=s_out, s_hist=hist, record=True, stream=stream)
    ctx._grad_token += 1
    return s_out.clone(), hist.clone(), ctx._grad_token, pr


def grad_backward(ctx: Context, problem, n_outer, u0, sbar_K, s_hist, token, y, b=None, stream=None):
    """Reverse sweep after grad_forward (problem = the problem' it returned,
    y and b = that forward's reference): uses that forward's records when no
    other grad_forward ran since (token), else recomputes from s_hist.  The
    context's copies of y and b are restored first (a later forward may have
    overwritten them)."""
    P, keep = problem
    n, m = MODEL_DIMS[P.model]
    T = P.T
    dev = u0.device
    _cached(ctx, "y", tuple(y.shape), torch.float32, dev).copy_(y)
    if b is not None:
        _cached(ctx, "b", tuple(b.shape), torch.float32, dev).copy_(b)
    if token == ctx._grad_token:
        hist = _cached(ctx, "hist", (max(int(n_outer), 1), T + 1, n), torch.float64, dev)
    else:
        hist = s_hist
    u0c = _cached(ctx, "bu0", (T, m), torch.float64, dev)
    sb = _cached(ctx, "bsbar", (T + 1, n), torch.float64, dev)
    u0c.copy_(u0)
    sb.copy_(sbar_K)
    mode = BACKWARD_CHECKPOINTS
    need = int(load().cov_workspace_size_backward(ctypes.byref(P), int(n_outer), mode))
    if need == 0:
        raise CovError(COV_ERR_UNSUPPORTED, "cov_solve_backward (Sinkhorn field, time-invariant model, d <= 3)")
    ctx.reserve(need)
    ybar = _cached(ctx, "ybar", (P.M, P.d), torch.float32, dev)
    bbar = _cached(ctx, "bbar", (P.M,), torch.float32, dev) if P.b else None
    s0bar = _cached(ctx, "s0bar", (n,), torch.float64, dev)
    u0bar = _cached(ctx, "u0bar", (T, m), torch.float64, dev)
    st = load().cov_solve_backward(ctx.h, ctypes.byref(P), int(n_outer), _ptr(u0c, torch.float64, (T, m), "u0"),
                                   _ptr(hist, torch.float64, name="s_hist"), _ptr(sb, torch.float64, (T + 1, n), "sbar"),
                                   _ptr(ybar, torch.float32, (P.M, P.d), "ybar"),
                                   _ptr(bbar, torch.float32, (P.M,), "bbar"), _ptr(s0bar, torch.float64, (n,), "s0bar"),
                                   _ptr(u0bar, torch.float64, (T, m), "u0bar"), _stream(stream))
    ctx._check(st, "cov_solve_backward")
    return ybar.clone(), (bbar.clone() if bbar is not None else None), s0bar.clone(), u0bar.clone()
