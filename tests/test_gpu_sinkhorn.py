"""GPU parity of the Sinkhorn-divergence field (Eq. 5-7) with the FP64 oracle.

Bars: potentials max|f_gpu - f_orc| / eps <= 1e-4; field norm-wise relative
error <= 1e-4 (FP32 path, exponentials through MUFU ex2.approx).  Inputs are
float32-exact so both sides see the same numbers.
"""
import numpy as np
import pytest
import torch

from conftest import dev32, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu

POT_TOL = 1e-4
FIELD_TOL = 1e-4

CASES = [  # T, M, d, eps, weighted
    (1, 1, 2, 0.05, False),
    (3, 5, 2, 0.05, True),
    (37, 53, 1, 0.02, False),
    (300, 517, 2, 0.01, True),
    (1000, 2100, 2, 0.005, False),
    (129, 257, 3, 0.02, True),
    (64, 100, 6, 0.1, False),
    (513, 300, 2, 0.005, True),
]


def _inputs(T, M, d, weighted, seed):
    x = wl.random_points(T, d, seed)
    y = wl.random_points(M, d, seed + 1)
    b = wl.random_weights(M, seed + 2) if weighted else None
    return x, y, b


@pytest.mark.parametrize("T,M,d,eps,weighted", CASES)
@pytest.mark.parametrize("n_iter", [0, 1, 6])
def test_fixed_iterations_match_oracle(cov, ctx, orc, T, M, d, eps, weighted, n_iter):
    x, y, b = _inputs(T, M, d, weighted, seed=T * 7 + M)
    a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(x), dev32(y), eps, n_iter, b=None if b is None else dev32(b))
    fo, go, po = orc.sinkhorn(x, y, b, eps, n_iter)
    ao = orc.sinkhorn_field(x, y, b, eps, go, po)
    assert np.abs(host(f) - fo).max() / eps <= POT_TOL
    assert np.abs(host(g) - go).max() / eps <= POT_TOL
    assert np.abs(host(p) - po).max() / eps <= POT_TOL
    assert rel_norm(host(a), ao) <= FIELD_TOL
    assert ctx.device_status()[1] == 0


@pytest.mark.parametrize("T,M,d,eps", [(300, 517, 3, 0.01), (200, 4099, 2, 0.02), (100, 2000, 5, 0.05)])
def test_reference_at_unaligned_addresses(cov, ctx, orc, T, M, d, eps):
    """The reference points and weights handed over one float past a 16-byte
    boundary (views into larger buffers): the reference statistics take their
    scalar path there, and the potentials and field still match the oracle."""
    x, y, b = _inputs(T, M, d, True, seed=11 * T + M)
    ybuf = torch.zeros(M * d + 4, dtype=torch.float32, device="cuda")
    bbuf = torch.zeros(M + 4, dtype=torch.float32, device="cuda")
    ybuf[1:1 + M * d] = dev32(y).reshape(-1)
    bbuf[1:1 + M] = dev32(b)
    yv, bv = ybuf[1:1 + M * d].view(M, d), bbuf[1:1 + M]
    assert yv.data_ptr() % 16 == 4 and bv.data_ptr() % 16 == 4
    a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(x), yv, eps, 6, b=bv)
    fo, go, po = orc.sinkhorn(x, y, b, eps, 6)
    ao = orc.sinkhorn_field(x, y, b, eps, go, po)
    for u, v in ((f, fo), (g, go), (p, po)):
        assert np.abs(host(u) - v).max() / eps <= POT_TOL
    assert rel_norm(host(a), ao) <= FIELD_TOL
    assert ctx.device_status()[1] == 0


@pytest.mark.parametrize("T,M,d,eps,weighted", CASES[2:6])
def test_single_update_from_identical_potentials(cov, ctx, orc, T, M, d, eps, weighted):
    """Teacher-forced: one GPU iteration from potentials the oracle produced
    (rounded to float32), against one oracle iteration from the same values."""
    x, y, b = _inputs(T, M, d, weighted, seed=T + 3 * M)
    fo, go, po = orc.sinkhorn(x, y, b, eps, 5)
    f0, g0, p0 = (v.astype(np.float32).astype(np.float64) for v in (fo, go, po))
    a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(x), dev32(y), eps, 1, b=None if b is None else dev32(b),
                                        f=dev32(f0), g=dev32(g0), p=dev32(p0), warm=True)
    f1, g1, p1 = orc.sinkhorn(x, y, b, eps, 1, f=f0, g=g0, p=p0)
    assert np.abs(host(g) - g1).max() / eps <= POT_TOL
    assert np.abs(host(f) - f1).max() / eps <= POT_TOL
    assert np.abs(host(p) - p1).max() / eps <= POT_TOL
    assert rel_norm(host(a), orc.sinkhorn_field(x, y, b, eps, g1, p1)) <= FIELD_TOL


def test_field_only_from_given_potentials(cov, ctx, orc):
    T, M, d, eps = 700, 900, 2, 0.01
    x, y, b = _inputs(T, M, d, True, seed=5)
    fo, go, po = orc.sinkhorn(x, y, b, eps, 10)
    f0, g0, p0 = (v.astype(np.float32).astype(np.float64) for v in (fo, go, po))
    a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(x), dev32(y), eps, 0, b=dev32(b), f=dev32(f0), g=dev32(g0),
                                        p=dev32(p0), warm=True)
    assert rel_norm(host(a), orc.sinkhorn_field(x, y, b, eps, g0, p0)) <= FIELD_TOL
    np.testing.assert_allclose(host(g), g0, atol=POT_TOL * eps)


@pytest.mark.parametrize("rows_per_thread", [2, 4, 8])
def test_tiling_options_give_the_same_answer(cov, ctx, orc, rows_per_thread):
    T, M, d, eps = 2049, 3001, 2, 0.01
    x, y, b = _inputs(T, M, d, False, seed=9)
    ctx.set_option(cov.OPT_ROWS_PER_THREAD, rows_per_thread)
    try:
        a, f, g, p = cov.cov_field_sinkhorn(ctx, dev32(x), dev32(y), eps, 3)
    finally:
        ctx.set_option(cov.OPT_ROWS_PER_THREAD, 4)
    fo, go, po = orc.sinkhorn(x, y, None, eps, 3)
    assert np.abs(host(f) - fo).max() / eps <= POT_TOL
    assert rel_norm(host(a), orc.sinkhorn_field(x, y, None, eps, go, po)) <= FIELD_TOL


def _sampled_rows_check(cov, ctx, orc, x, y, eps, warm_iters, n_rows, seed):
    """Run `warm_iters` iterations, then one more from the GPU's own
    potentials; recompute sampled rows of each update and of the field with
    the oracle from those same inputs (exact: a row depends only on the other
    side's potentials and points)."""
    T, M = len(x), len(y)
    X, Y = dev32(x), dev32(y)
    _, f, g, p = cov.cov_field_sinkhorn(ctx, X, Y, eps, warm_iters, field=False)
    fin, gin, pin = host(f), host(g), host(p)
    a, f1, g1, p1 = cov.cov_field_sinkhorn(ctx, X, Y, eps, 1, f=f.clone(), g=g.clone(), p=p.clone(), warm=True)
    torch.cuda.synchronize()
    rng = wl.rng(seed)
    ry = np.sort(rng.choice(M, size=min(n_rows, M), replace=False))
    rx = np.sort(rng.choice(T, size=min(n_rows, T), replace=False))
    g1h, f1h, p1h = host(g1), host(f1), host(p1)
    ge = np.abs(orc.sinkhorn_g_update(x, y, eps, fin, rows=ry) - g1h[ry]).max() / eps
    fe = np.abs(orc.sinkhorn_f_update(x, y, None, eps, g1h, rows=rx) - f1h[rx]).max() / eps
    pe = np.abs(orc.sinkhorn_p_update(x, eps, pin, rows=rx) - p1h[rx]).max() / eps
    ae = rel_norm(host(a)[rx], orc.sinkhorn_field(x, y, None, eps, g1h, p1h, rows=rx))
    assert ctx.device_status()[1] == 0
    return ge, fe, pe, ae


def test_full_size_double_integrator_workload_sampled_rows(cov, ctx, orc):
    """T = 4096, M = 16384, eps = 0.005 (the benchmark workload's field)."""
    inst = wl.make_instance(wl.SINKHORN_DOUBLE_T4096)
    w = inst.wl
    s = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    x = wl.f32_pair(s[1:, :2])[1]
    errs = _sampled_rows_check(cov, ctx, orc, x, inst.y, w.eps, w.n_iter - 1, 512, seed=1)
    assert max(errs[:3]) <= POT_TOL, errs
    assert errs[3] <= FIELD_TOL, errs


def _cold_iteration_check(cov, ctx, orc, x, y, eps, k, n_rows, seed, field):
    """Iteration k of a cold-start field evaluation (the schedule the solve
    runs), checked on sampled rows: the GPU's state after k - 1 iterations
    (zeros for k = 1) is the input, its state after k iterations the output,
    and the oracle recomputes the sampled rows of the g-, f- and p-updates of
    iteration k from the GPU's own inputs (g from f^(k-1), f from the new g,
    p from p^(k-1)) and, with `field`, the sampled rows of the Eq. 7 field
    from the final g and p.  Exact per row: a row depends only on the other
    side's potentials and the points."""
    T, M = len(x), len(y)
    X, Y = dev32(x), dev32(y)
    if k == 1:
        fin, pin = np.zeros(T), np.zeros(T)
    else:
        _, f0, _, p0 = cov.cov_field_sinkhorn(ctx, X, Y, eps, k - 1, field=False)
        fin, pin = host(f0), host(p0)
    a, f1, g1, p1 = cov.cov_field_sinkhorn(ctx, X, Y, eps, k, field=field)
    torch.cuda.synchronize()
    rng = wl.rng(seed)
    ry = np.sort(rng.choice(M, size=min(n_rows, M), replace=False))
    rx = np.sort(rng.choice(T, size=min(n_rows, T), replace=False))
    g1h, f1h, p1h = host(g1), host(f1), host(p1)
    ge = np.abs(orc.sinkhorn_g_update(x, y, eps, fin, rows=ry) - g1h[ry]).max() / eps
    fe = np.abs(orc.sinkhorn_f_update(x, y, None, eps, g1h, rows=rx) - f1h[rx]).max() / eps
    pe = np.abs(orc.sinkhorn_p_update(x, eps, pin, rows=rx) - p1h[rx]).max() / eps
    ae = rel_norm(host(a)[rx], orc.sinkhorn_field(x, y, None, eps, g1h, p1h, rows=rx)) if field else 0.0
    assert ctx.device_status()[1] == 0
    return ge, fe, pe, ae


@pytest.fixture(scope="module")
def unicycle_density_inputs(orc):
    inst = wl.make_instance(wl.SINKHORN_UNICYCLE_T65536)
    w = inst.wl
    s = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    return wl.f32_pair(s[1:, :2])[1], inst.y, w


@pytest.mark.parametrize("k", [1, 50, 100])
def test_full_size_unicycle_density_workload_iterations(cov, ctx, orc, unicycle_density_inputs, k):
    """T = 65536, M = 262144, eps = 0.002 (density-map reference), iterations
    1, n_iter/2 and n_iter of the 100-iteration cold schedule on the default
    exponent path (at this size the fixed-offset iterations 2..100 take the
    tensor-core kernel; iteration 1 the running-maximum CUDA-core form), 4096
    sampled rows of every update and, at iteration 100, of the field."""
    x, y, w = unicycle_density_inputs
    assert k <= w.n_iter
    errs = _cold_iteration_check(cov, ctx, orc, x, y, w.eps, k, 4096, seed=10 + k, field=k == w.n_iter)
    assert max(errs[:3]) <= POT_TOL, errs
    assert errs[3] <= FIELD_TOL, errs


def test_full_size_unicycle_density_workload_warm_update(cov, ctx, orc, unicycle_density_inputs):
    """The same workload, one warm-started iteration after three cold ones."""
    x, y, w = unicycle_density_inputs
    errs = _sampled_rows_check(cov, ctx, orc, x, y, w.eps, 3, 128, seed=2)
    assert max(errs[:3]) <= POT_TOL, errs
    assert errs[3] <= FIELD_TOL, errs


def test_full_size_field_is_permutation_equivariant(cov, ctx, unicycle_density_inputs):
    """A property that holds at any size, checked on the whole field at
    T = 65536, M = 262144 and 100 iterations on the default path: relabelling
    the reference samples leaves the field unchanged and relabelling the
    trajectory points relabels it (each within the field's parity bar; the
    sums run in another order)."""
    x, y, w = unicycle_density_inputs
    xd, yd = dev32(x), dev32(y)
    a = host(cov.cov_field_sinkhorn(ctx, xd, yd, w.eps, w.n_iter)[0])
    rng = np.random.default_rng(11)
    px, py = rng.permutation(len(x)), rng.permutation(len(y))
    a_y = host(cov.cov_field_sinkhorn(ctx, xd, dev32(y[py]), w.eps, w.n_iter)[0])
    assert rel_norm(a_y, a) <= FIELD_TOL
    a_x = host(cov.cov_field_sinkhorn(ctx, dev32(x[px]), yd, w.eps, w.n_iter)[0])
    assert rel_norm(a_x, a[px]) <= FIELD_TOL
    assert ctx.device_status()[1] == 0


def test_repeated_calls_are_bitwise_identical(cov, ctx):
    """Column splits are merged in split order (no float atomics), so the
    same inputs give the same bits, at a size with 30+ splits per row block."""
    T, M, eps = 4096, 16384, 0.005
    x, y, b = _inputs(T, M, 2, True, seed=77)
    xd, yd, bd = dev32(x), dev32(y), dev32(b)
    r1 = [host(t) for t in cov.cov_field_sinkhorn(ctx, xd, yd, eps, 8, b=bd)]
    r2 = [host(t) for t in cov.cov_field_sinkhorn(ctx, xd, yd, eps, 8, b=bd)]
    for u, v in zip(r1, r2):
        np.testing.assert_array_equal(u, v)
    assert ctx.device_status()[1] == 0
