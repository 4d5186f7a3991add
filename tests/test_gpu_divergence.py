"""GPU parity of cov_sinkhorn_divergence (Eq. 6 value at n_iter fixed
iterations, and its envelope gradient -(1/T) field of Eq. 7) with the FP64
oracle.

Bars: the value is <a, f> + <b, g> - <a, p> - <b, q> of four potentials each
within 1e-4 eps of the oracle's, so |S_gpu - S_orc| <= 4e-4 eps; the
gradient is the field scaled by -1/T, norm-wise 1e-4 like the field."""
import numpy as np
import pytest
import torch

from conftest import dev32, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("T,M,eps,n_iter", [(1, 1, 0.05, 3), (300, 517, 0.02, 10), (2048, 4096, 0.005, 100)])
def test_value_and_gradient_match_oracle(cov, ctx, orc, T, M, eps, n_iter):
    x = wl.random_points(T, 2, seed=T + 1)
    y = wl.random_points(M, 2, seed=M + 2, lo=0.1, hi=0.9)
    value, grad, q = cov.cov_sinkhorn_divergence(ctx, dev32(x), dev32(y), eps, n_iter)
    torch.cuda.synchronize()
    So = orc.sinkhorn_divergence_iter(x, y, eps, n_iter)
    assert abs(float(value) - So) <= 4e-4 * eps, (float(value), So)
    _, go, po = orc.sinkhorn(x, y, None, eps, n_iter)
    gref = -orc.sinkhorn_field(x, y, None, eps, go, po) / T
    assert rel_norm(host(grad), gref) <= 1e-4
    qo = orc.sinkhorn(y, y, None, eps, n_iter)[2]
    assert np.abs(host(q) - qo).max() / eps <= 1e-4
    assert ctx.device_status() == (cov.COV_OK, 0)


def test_given_reference_potential_is_reused(cov, ctx):
    """A call with q_given reads the reference self potential of an earlier
    call instead of recomputing it, and gives the value a fresh call gives."""
    eps, n = 0.01, 12
    y = dev32(wl.random_points(700, 2, seed=5))
    x1 = dev32(wl.random_points(400, 2, seed=6))
    x2 = dev32(wl.random_points(333, 2, seed=7))
    _, _, q = cov.cov_sinkhorn_divergence(ctx, x1, y, eps, n, grad=False)
    v_given, g_given, _ = cov.cov_sinkhorn_divergence(ctx, x2, y, eps, n, q_ref=q, q_given=True)
    v_fresh, g_fresh, _ = cov.cov_sinkhorn_divergence(ctx, x2, y, eps, n)
    torch.cuda.synchronize()
    assert float(v_given) == float(v_fresh)
    np.testing.assert_array_equal(host(g_given), host(g_fresh))


def test_weighted_reference_needs_its_self_potential(cov, ctx):
    x = dev32(wl.random_points(50, 2, seed=8))
    y = dev32(wl.random_points(60, 2, seed=9))
    b = dev32(wl.random_weights(60, seed=10))
    with pytest.raises(cov.CovError) as e:
        cov.cov_sinkhorn_divergence(ctx, x, y, 0.05, 3, b=b)
    assert e.value.status == cov.COV_ERR_UNSUPPORTED
    q = torch.zeros(60, device="cuda", dtype=torch.float32)
    v, g, _ = cov.cov_sinkhorn_divergence(ctx, x, y, 0.05, 3, b=b, q_ref=q, q_given=True)
    torch.cuda.synchronize()
    assert np.isfinite(float(v)) and np.isfinite(host(g)).all()
