"""GPU parity of the tensor-core exponent path of the Sinkhorn updates.

From the third iteration (or at once from a warm start) every update runs
with a fixed row offset; for d <= 3 its exponents w_ij - o_i come from
tcgen05 kind::tf32 MMAs on TF32-split operands instead of FP32 FMAs.  The
bars are those of the plain field (potentials max|f - f_orc| / eps <= 1e-4,
field norm-wise 1e-4): the split keeps every product exact and the tensor
core's FP32 accumulation adds an error of about 1e-5 bits per exponent at
these magnitudes, below the MUFU ex2.approx error budget the bars allow.
The CUDA-core path (COV_OPT_TENSOR_CORES = 0; the default, 2, takes it for
launches under 2^30 pairs) is held to the same bars, and the two paths to
each other.
"""
import numpy as np
import pytest

from conftest import dev32, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu

POT_TOL = 1e-4
FIELD_TOL = 1e-4

CASES = [  # T, M, d, eps, weighted, n_iter
    (1, 1, 2, 0.05, False, 5),
    (37, 53, 1, 0.02, False, 8),
    (129, 257, 3, 0.02, True, 8),
    (300, 517, 2, 0.01, True, 12),
    (1000, 2100, 2, 0.005, False, 10),
    (2049, 3001, 2, 0.002, True, 6),     # eps of the large workload: exponent terms up to ~1e3 bits
    (4096, 700, 3, 0.01, False, 6),      # many row blocks, few columns
    (130, 9000, 1, 0.01, True, 6),       # two row blocks, many column splits
]


def _run(cov, ctx, x, y, b, eps, n_iter, tc, **kw):
    ctx.set_option(cov.OPT_TENSOR_CORES, tc)
    try:
        out = cov.cov_field_sinkhorn(ctx, dev32(x), dev32(y), eps, n_iter, b=None if b is None else dev32(b), **kw)
    finally:
        ctx.set_option(cov.OPT_TENSOR_CORES, cov.TENSOR_CORES_AUTO)
    st, flags = ctx.device_status()
    assert st == cov.COV_OK, flags
    return out


@pytest.mark.parametrize("T,M,d,eps,weighted,n_iter", CASES)
@pytest.mark.parametrize("tc", [1, 0])
def test_fixed_offset_iterations_match_oracle(cov, ctx, orc, T, M, d, eps, weighted, n_iter, tc):
    x = wl.random_points(T, d, seed=901 + T)
    y = wl.random_points(M, d, seed=902 + M)
    b = wl.random_weights(M, seed=903) if weighted else None
    a, f, g, p = _run(cov, ctx, x, y, b, eps, n_iter, tc)
    fo, go, po = orc.sinkhorn(x, y, b, eps, n_iter)
    for u, v in ((f, fo), (g, go), (p, po)):
        assert np.abs(host(u) - v).max() / eps <= POT_TOL
    assert rel_norm(host(a), orc.sinkhorn_field(x, y, b, eps, go, po)) <= FIELD_TOL


@pytest.mark.parametrize("T,M,d,eps", [(300, 517, 2, 0.01), (129, 257, 3, 0.02), (37, 53, 1, 0.02)])
def test_warm_single_iteration_is_all_tensor_core(cov, ctx, orc, T, M, d, eps):
    """From warm potentials the first iteration's three updates all take the
    fixed-offset path (the p-update with its fixed-point offset)."""
    x = wl.random_points(T, d, seed=911)
    y = wl.random_points(M, d, seed=912)
    fo, go, po = orc.sinkhorn(x, y, None, eps, 20)
    f0, g0, p0 = (wl.f32_pair(v)[1] for v in (fo, go, po))
    a, f, g, p = _run(cov, ctx, x, y, None, eps, 1, 1, f=dev32(f0), g=dev32(g0), p=dev32(p0), warm=True)
    f1, g1, p1 = orc.sinkhorn(x, y, None, eps, 1, f=f0, g=g0, p=p0)
    for u, v in ((f, f1), (g, g1), (p, p1)):
        assert np.abs(host(u) - v).max() / eps <= POT_TOL
    assert rel_norm(host(a), orc.sinkhorn_field(x, y, None, eps, g1, p1)) <= FIELD_TOL


def test_tensor_core_and_cuda_core_paths_agree_at_full_size(cov, ctx):
    """T = 4096, M = 16384, eps = 0.005, 30 iterations: the two exponent
    paths give the same potentials within the parity bar (each is held to
    the oracle above and, row-sampled, at this size in the field tests)."""
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096)
    x = wl.random_points(4096, 2, seed=921, lo=0.1, hi=0.9)
    y = inst.y
    r1 = _run(cov, ctx, x, y, None, inst.wl.eps, 30, 1)
    r0 = _run(cov, ctx, x, y, None, inst.wl.eps, 30, 0)
    for u, v in zip(r1[1:], r0[1:]):
        assert np.abs(host(u) - host(v)).max() / inst.wl.eps <= POT_TOL
    assert rel_norm(host(r1[0]), host(r0[0])) <= FIELD_TOL


def test_full_size_double_integrator_workload_sampled_rows_tensor_cores(cov, ctx, orc):
    """T = 4096, M = 16384, eps = 0.005 on the tensor-core path: 49
    iterations, then one more from the GPU's own potentials (all three
    updates with fixed offsets), sampled rows recomputed by the oracle."""
    from test_gpu_sinkhorn import _sampled_rows_check
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096)
    w = inst.wl
    s = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    x = wl.f32_pair(s[1:, :2])[1]
    ctx.set_option(cov.OPT_TENSOR_CORES, 1)
    try:
        errs = _sampled_rows_check(cov, ctx, orc, x, inst.y, w.eps, w.n_iter - 1, 512, seed=3)
    finally:
        ctx.set_option(cov.OPT_TENSOR_CORES, cov.TENSOR_CORES_AUTO)
    assert max(errs[:3]) <= POT_TOL, errs
    assert errs[3] <= FIELD_TOL, errs


def test_option_is_validated(cov, ctx):
    with pytest.raises(cov.CovError):
        ctx.set_option(cov.OPT_TENSOR_CORES, 3)


def test_fma_pipe_exp2_accuracy_and_rate(cov, ctx):
    """2^x on the FMA pipe (the alternative to MUFU ex2 the tensor-core
    kernel can take for part of its exponentials): largest relative error
    against FP64 exp2 on [-125, 127] within 3e-7 (its degree-5 Chebyshev
    fit is 1.0e-7 in exact arithmetic, 2.4e-7 evaluated in FP32; MUFU
    ex2.approx is of the same order), and both rates are measured."""
    pr = cov.cov_probe_peaks(ctx, 256)
    assert 0.0 < pr["exp2_fma_max_rel_err"] <= 3e-7, pr
    assert pr["exp2_fma_values_s"] > 0 and pr["ex2_lane_ops_s"] > 0
