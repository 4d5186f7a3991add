"""Argument checking, workspace errors and device status of the C-ABI."""
import ctypes

import numpy as np
import pytest
import torch

from conftest import dev32, dev64, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_invalid_arguments_are_rejected_without_launching(cov, ctx):
    x = dev32(wl.random_points(10, 2, 1))
    y = dev32(wl.random_points(12, 2, 2))
    with pytest.raises(cov.CovError) as e:
        cov.cov_field_sinkhorn(ctx, x, y, 0.0, 3)
    assert e.value.status == cov.COV_ERR_INVALID_ARG
    with pytest.raises(cov.CovError):
        cov.cov_field_sinkhorn(ctx, x, y, 0.1, -1)
    with pytest.raises(cov.CovError):
        cov.cov_field_svgd(ctx, x, -1.0, score=x)
    x7 = dev32(wl.random_points(10, 7, 1))
    with pytest.raises(cov.CovError):
        cov.cov_field_svgd(ctx, x7, 0.1, score=x7)
    L = cov.load()
    st = L.cov_field_sinkhorn(ctx.h, ctypes.c_void_p(x.data_ptr()), 10, ctypes.c_void_p(y.data_ptr()), None, 12, 2,
                              ctypes.c_float(0.1), 1, cov.WARM_START, None, None, None, None, None)
    assert st == cov.COV_ERR_INVALID_ARG
    assert ctx.device_status() == (cov.COV_OK, 0)


def test_workspace_too_small(cov):
    c = cov.Context(0, workspace_bytes=1024)
    try:
        x = dev32(wl.random_points(100, 2, 1))
        out = torch.empty_like(x)
        L = cov.load()
        st = L.cov_field_svgd(c.h, ctypes.c_void_p(x.data_ptr()), 100, 2, ctypes.c_void_p(x.data_ptr()), None,
                              ctypes.c_float(0.1), ctypes.c_void_p(out.data_ptr()), None)
        assert st == cov.COV_ERR_WORKSPACE
    finally:
        c.close()


def test_nonfinite_input_sets_status(cov, ctx):
    x = wl.random_points(50, 2, 1)
    x[3, 0] = np.nan
    cov.cov_field_sinkhorn(ctx, dev32(x), dev32(wl.random_points(60, 2, 2)), 0.05, 2)
    st, fl = ctx.device_status()
    assert fl & cov.DEV_NONFINITE and st == cov.COV_ERR_NONFINITE
    assert ctx.device_status() == (cov.COV_OK, 0)   # read clears


@pytest.mark.parametrize("T", [50, 2000])
def test_stein_field_nonfinite_and_empty(cov, ctx, T):
    """A NaN coordinate sets the non-finite status on both Stein paths (the
    one-launch kernel up to T = 1024, the all-pairs kernel above); an empty
    trajectory is an argument error."""
    x = wl.random_points(T, 2, 5)
    x[T // 2, 1] = np.nan
    w, mu, sigma = (wl.f32_pair(v)[1] for v in wl.gmm_params(3, seed=2, d=2))
    cov.cov_field_svgd(ctx, dev32(x), 0.05, gmm=(w, mu, sigma))
    st, fl = ctx.device_status()
    assert fl & cov.DEV_NONFINITE and st == cov.COV_ERR_NONFINITE
    assert ctx.device_status() == (cov.COV_OK, 0)
    xd = dev32(wl.random_points(4, 2, 1))
    out = torch.empty_like(xd)
    L = cov.load()
    st = L.cov_field_svgd(ctx.h, ctypes.c_void_p(xd.data_ptr()), 0, 2, ctypes.c_void_p(xd.data_ptr()), None,
                          ctypes.c_float(0.1), ctypes.c_void_p(out.data_ptr()), None)
    assert st == cov.COV_ERR_INVALID_ARG


@pytest.mark.parametrize("tensor_cores", [0, 1])
@pytest.mark.parametrize("n_iter", [1, 4])
def test_bounded_wait_gives_up_and_reports_timeout(cov, ctx, orc, n_iter, tensor_cores):
    """A wait limit of zero polls makes every tile wait give up at once; the
    kernel drains its copies (and, in the tensor-core kernel that the fixed-
    offset iterations 2.. run on when tensor_cores = 1, its MMAs, before it
    frees its tensor memory) with a limit of its own, raises the timeout bit
    and returns, and the context stays usable: the next call on the same
    exponent path matches the oracle."""
    x = wl.random_points(300, 2, 1)
    y = wl.random_points(400, 2, 2)
    ctx.set_option(cov.OPT_TENSOR_CORES, tensor_cores)
    try:
        ctx.set_option(cov.OPT_SPIN_LIMIT, 0)
        try:
            cov.cov_field_sinkhorn(ctx, dev32(x), dev32(y), 0.05, n_iter)
            st, fl = ctx.device_status()
        finally:
            ctx.set_option(cov.OPT_SPIN_LIMIT, 1 << 22)
        assert fl & cov.DEV_TIMEOUT and st == cov.COV_ERR_TIMEOUT
        a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(x), dev32(y), 0.05, n_iter)
        fo, go, po = orc.sinkhorn(x, y, None, 0.05, n_iter)
        for u, v in ((f, fo), (g, go), (p, po)):
            assert np.abs(host(u) - v).max() / 0.05 <= 1e-4
        assert rel_norm(host(a), orc.sinkhorn_field(x, y, None, 0.05, go, po)) <= 1e-4
        assert ctx.device_status() == (cov.COV_OK, 0)
    finally:
        ctx.set_option(cov.OPT_TENSOR_CORES, cov.TENSOR_CORES_AUTO)


def test_ragged_and_degenerate_sizes(cov, ctx, orc):
    # identical points: field zero by symmetry of the debiased divergence
    x = wl.random_points(33, 2, 4)
    a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(x), dev32(x), 0.05, 200)
    assert np.abs(host(a)).max() < 1e-3
    # every trajectory point at the same place, one reference point
    xs = np.tile([[0.25, 0.75]], (17, 1))
    a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(xs), dev32(np.array([[0.5, 0.25]])), 0.01, 3)
    np.testing.assert_allclose(host(a), np.tile(2 * (np.array([0.5, 0.25]) - [0.25, 0.75]), (17, 1)), rtol=1e-5)


def test_autotuner_sweeps_and_applies_a_tile_shape(cov, orc, tmp_path):
    """cov_autotune_sinkhorn times every candidate, applies the fastest, and
    the field computed with the tuned shape still matches the oracle; the
    Python cache round-trips the choice."""
    from paper_2511_11514_b300 import autotune
    T, M, eps = 2048, 4096, 0.01
    x = wl.random_points(T, 2, seed=901)
    y = wl.random_points(M, 2, seed=902)
    ctx = cov.Context(0)
    try:
        R, cps, rows = cov.cov_autotune_sinkhorn(ctx, dev32(x), dev32(y), eps)
        assert (R, cps) in [(r[0], r[1]) for r in rows]
        assert all(r[2] > 0 for r in rows)
        assert min(rows, key=lambda r: r[2])[:2] == (R, cps)
        a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(x), dev32(y), eps, 5)
        fo, go, po = orc.sinkhorn(x, y, None, eps, 5)
        assert np.abs(host(f) - fo).max() / eps <= 1e-4
        ch = autotune.tune_sinkhorn(ctx, dev32(x), dev32(y), eps, cache_path=str(tmp_path / "c.json"))
        ch2 = autotune.tune_sinkhorn(ctx, dev32(x), dev32(y), eps, cache_path=str(tmp_path / "c.json"))
        assert (ch["R"], ch["ctas_per_sm"]) == (ch2["R"], ch2["ctas_per_sm"])
    finally:
        ctx.close()
