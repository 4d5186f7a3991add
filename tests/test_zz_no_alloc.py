"""cov_field_sinkhorn_noalloc against cov_field_sinkhorn and the oracle.

The no-allocation entry point exists for programs that may not call
cudaMalloc: plugins whose host application owns all device memory and hands
it out from its own arena, or real-time loops that cannot take the
device-wide synchronisation cudaMalloc/cudaFree imply.  It keeps its scratch
in one fixed 48 MiB array inside the library.  Two calls in a row -- the
second on other sizes, so it starts from whatever the first left in the
shared array -- must give the results of the regular entry point with a
context workspace, within the parity tolerances used everywhere else
(potentials 1e-4 eps, field 1e-4 norm-wise); at the largest workload it
states it takes (T = 65536, M = 262144) it must match the FP64 oracle on
sampled rows, and one reference point past its capacity it must refuse the
call.  This file is collected last on purpose.
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


def _field_noalloc(cov, x, y, eps, n_iter):
    T, d = x.shape
    M = y.shape[0]
    f = torch.empty(T, device="cuda", dtype=torch.float32)
    g = torch.empty(M, device="cuda", dtype=torch.float32)
    p = torch.empty(T, device="cuda", dtype=torch.float32)
    a = torch.empty_like(x)
    st = cov.load().cov_field_sinkhorn_noalloc(
        _p(x), T, _p(y), None, M, d, ctypes.c_float(eps), n_iter, 0, _p(f), _p(g), _p(p), _p(a),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, a, f, g, p


def test_noalloc_at_its_largest_stated_workload_matches_the_oracle(cov, orc):
    """T = 65536 trajectory points of the unicycle workload's initial
    rollout, M = 262144 density-map samples, eps = 0.002: two calls in a row
    (2 and 3 iterations; the fixed-offset third iteration runs on the
    tensor-core kernel at this size), and the third iteration's g-, f- and
    p-updates and the field recomputed by the oracle on 1024 sampled rows from
    the second call's inputs (exact per row)."""
    inst = wl.make_instance(wl.SINKHORN_UNICYCLE_T65536)
    w = inst.wl
    s = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    x = wl.f32_pair(s[1:, :2])[1]
    y = inst.y
    T, M, eps = len(x), len(y), w.eps
    assert (T, M) == (65536, 262144)
    X = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(y, dtype=torch.float32, device="cuda")
    st, _, f2, _, p2 = _field_noalloc(cov, X, Y, eps, 2)
    assert st == cov.COV_OK, cov.status_string(st)
    st, a3, f3, g3, p3 = _field_noalloc(cov, X, Y, eps, 3)
    assert st == cov.COV_OK, cov.status_string(st)
    torch.cuda.synchronize()
    rng = wl.rng(31)
    ry = np.sort(rng.choice(M, size=1024, replace=False))
    rx = np.sort(rng.choice(T, size=1024, replace=False))
    f2h, p2h, f3h, g3h, p3h = (_h(t) for t in (f2, p2, f3, g3, p3))
    assert np.abs(orc.sinkhorn_g_update(x, y, eps, f2h, rows=ry) - g3h[ry]).max() / eps <= POT_TOL
    assert np.abs(orc.sinkhorn_f_update(x, y, None, eps, g3h, rows=rx) - f3h[rx]).max() / eps <= POT_TOL
    assert np.abs(orc.sinkhorn_p_update(x, eps, p2h, rows=rx) - p3h[rx]).max() / eps <= POT_TOL
    ao = orc.sinkhorn_field(x, y, None, eps, g3h, p3h, rows=rx)
    assert np.linalg.norm(_h(a3)[rx] - ao) <= FIELD_TOL * np.linalg.norm(ao)


def test_noalloc_capacity_boundary(cov):
    """At T = 65536, d = 2 the array holds the scratch of up to M = 347136
    reference points: that call runs (and agrees with the workspace entry
    point), one point more is refused with COV_ERR_WORKSPACE before anything
    is launched."""
    T, eps = 65536, 0.01
    x = torch.as_tensor(wl.random_points(T, 2, 41), dtype=torch.float32, device="cuda")
    ctx = cov.Context(0)
    try:
        for M, ok in ((347136, True), (347137, False)):
            y = torch.as_tensor(wl.random_points(M, 2, 42), dtype=torch.float32, device="cuda")
            st, a1, f1, g1, p1 = _field_noalloc(cov, x, y, eps, 1)
            torch.cuda.synchronize()
            if not ok:
                assert st == cov.COV_ERR_WORKSPACE, cov.status_string(st)
                continue
            assert st == cov.COV_OK, cov.status_string(st)
            a0, f0, g0, p0 = cov.cov_field_sinkhorn(ctx, x, y, eps, 1)
            torch.cuda.synchronize()
            for u, v in ((f1, f0), (g1, g0), (p1, p0)):
                assert np.abs(_h(u) - _h(v)).max() / eps <= POT_TOL
            assert np.linalg.norm(_h(a1) - _h(a0)) <= FIELD_TOL * np.linalg.norm(_h(a0))
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
