"""cov_field_sinkhorn_noalloc against cov_field_sinkhorn.

The no-allocation entry point exists for programs that may not call
cudaMalloc (for example while a CUDA graph is being captured, inside a plugin
whose host owns all device memory, or in a real-time loop that cannot take
the synchronisation cudaMalloc/cudaFree imply).  It keeps its scratch in one
fixed array inside the library.  Two calls in a row -- the second on other
sizes, so it starts from whatever the first left in the shared array -- must
give the results of the regular entry point with a context workspace, within
the parity tolerances used everywhere else (potentials 1e-4 eps, field 1e-4
norm-wise).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu

POT_TOL = 1e-4
FIELD_TOL = 1e-4


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _noalloc(cov, x, y, eps, n_iter, b=None):
    T, d = x.shape
    M = y.shape[0]
    f = torch.empty(T, device="cuda", dtype=torch.float32)
    g = torch.empty(M, device="cuda", dtype=torch.float32)
    p = torch.empty(T, device="cuda", dtype=torch.float32)
    a = torch.empty_like(x)
    st = cov.load().cov_field_sinkhorn_noalloc(
        _p(x), T, _p(y), _p(b), M, d, ctypes.c_float(eps), n_iter, 0, _p(f), _p(g), _p(p), _p(a),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == cov.COV_OK, cov.status_string(st)
    return a, f, g, p


def _h(t):
    return t.detach().cpu().double().numpy()


def test_noalloc_matches_the_workspace_entry_point_twice_in_a_row(cov):
    ctx = cov.Context(0)
    try:
        cases = [(1000, 2100, 2, 0.005, 6, True, 1), (300, 517, 3, 0.02, 3, False, 2)]
        for T, M, d, eps, n_iter, weighted, seed in cases:
            x = torch.as_tensor(wl.random_points(T, d, seed), dtype=torch.float32, device="cuda")
            y = torch.as_tensor(wl.random_points(M, d, seed + 1), dtype=torch.float32, device="cuda")
            b = (torch.as_tensor(wl.random_weights(M, seed + 2), dtype=torch.float32, device="cuda")
                 if weighted else None)
            a1, f1, g1, p1 = _noalloc(cov, x, y, eps, n_iter, b)
            a0, f0, g0, p0 = cov.cov_field_sinkhorn(ctx, x, y, eps, n_iter, b=b)
            torch.cuda.synchronize()
            for u, v in ((f1, f0), (g1, g0), (p1, p0)):
                assert np.abs(_h(u) - _h(v)).max() / eps <= POT_TOL
            assert np.linalg.norm(_h(a1) - _h(a0)) <= FIELD_TOL * np.linalg.norm(_h(a0))
            assert np.isfinite(_h(a1)).all()
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array(cov):
    n = 1 << 22
    x = torch.zeros((n, 2), device="cuda", dtype=torch.float32)
    f = torch.empty(n, device="cuda", dtype=torch.float32)
    st = cov.load().cov_field_sinkhorn_noalloc(
        _p(x), n, _p(x), None, n, 2, ctypes.c_float(0.01), 1, 0, _p(f), _p(f), _p(f), _p(x),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == cov.COV_ERR_WORKSPACE
