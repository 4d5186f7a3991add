"""GPU parity of the Stein field's reverse mode (cov_field_svgd_vjp, Eq. 4)
with the FP64 oracle's reverse mode (itself pinned by central differences).

Bar: norm-wise relative error 1e-4 for every gradient (the field's own bar;
the reverse pass is one FP32 all-pairs sum with MUFU exponentials, and the
mixture gradients are FP64 sums of FP32 per-point terms)."""
import numpy as np
import pytest
import torch

from conftest import dev32, host, rel_norm
from paper_2511_11514_b300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.mark.parametrize("T,d,h", [(1, 2, 0.1), (37, 1, 0.2), (300, 2, 0.05), (1000, 3, 0.1), (4099, 2, 0.05),
                                   (129, 6, 0.4)])
def test_vjp_with_given_score_matches_oracle(cov, ctx, orc, T, d, h):
    rng = wl.rng(1000 + T + d)
    x = wl.f32_pair(rng.uniform(0, 1, size=(T, d)))[1]
    s = wl.f32_pair(rng.standard_normal((T, d)) * 5.0)[1]
    ab = wl.f32_pair(rng.standard_normal((T, d)))[1]
    xb, sb = cov.cov_field_svgd_vjp(ctx, dev32(x), h, dev32(ab), score=dev32(s))
    xo, so = orc.svgd_field_vjp(x, s, h, ab)
    if T == 1:
        assert np.abs(host(xb)).max() == 0.0
    else:
        assert rel_norm(host(xb), xo) <= TOL
    assert rel_norm(host(sb), so) <= TOL
    assert ctx.device_status() == (cov.COV_OK, 0)


@pytest.mark.parametrize("T,K,h,seed", [(256, 3, 0.05, 0), (1000, 16, 0.05, 3), (2049, 8, 0.08, 5)])
def test_vjp_through_the_mixture_score_matches_oracle(cov, ctx, orc, T, K, h, seed):
    """Total gradient in x (kernel and score paths) and the mixture
    gradients, on trajectories of the Stein workload's shape (a noisy line
    through the unit square) and mixtures of its generator."""
    s0, u0 = wl.line_controls_single(T, 0.1, seed)
    x = wl.f32_pair(orc.rollout(wl.SINGLE_INT, s0, u0, 0.1)[1:])[1]
    gmm = tuple(wl.f32_pair(v)[1] for v in wl.gmm_params(K, seed=seed))
    ab = wl.f32_pair(wl.rng(seed + 7).standard_normal((T, 2)))[1]
    xb, sb, (wb, mb, sgb) = cov.cov_field_svgd_vjp(ctx, dev32(x), h, dev32(ab), gmm=gmm)
    xo, wo, mo, so = orc.svgd_gmm_field_vjp(x, *gmm, h, ab)
    assert rel_norm(host(xb), xo) <= TOL
    assert rel_norm(host(mb), mo) <= TOL
    assert rel_norm(host(sgb), so) <= TOL
    assert rel_norm(host(wb), wo) <= TOL
    # the score cotangent is the fixed-score reverse mode's sbar
    _, sbo = orc.svgd_field_vjp(x, orc.gmm_score(x, *gmm), h, ab)
    assert rel_norm(host(sb), sbo) <= TOL
    assert ctx.device_status() == (cov.COV_OK, 0)


def test_vjp_is_deterministic_and_rejects_bad_arguments(cov, ctx):
    x = dev32(wl.random_points(777, 2, seed=3))
    ab = dev32(wl.rng(4).standard_normal((777, 2)))
    gmm = tuple(wl.f32_pair(v)[1] for v in wl.gmm_params(5, seed=2))
    r1 = cov.cov_field_svgd_vjp(ctx, x, 0.07, ab, gmm=gmm)
    r2 = cov.cov_field_svgd_vjp(ctx, x, 0.07, ab, gmm=gmm)
    for u, v in zip(r1[:2] + r1[2], r2[:2] + r2[2]):
        np.testing.assert_array_equal(host(u), host(v))
    with pytest.raises(cov.CovError) as e:
        cov.cov_field_svgd_vjp(ctx, x, 0.0, ab, gmm=gmm)
    assert e.value.status == cov.COV_ERR_INVALID_ARG


@pytest.mark.parametrize("T,d,K", [(700, 3, 32), (257, 6, 7), (64, 1, 2)])
def test_vjp_through_mixture_in_other_dimensions(cov, ctx, orc, T, d, K):
    """The mixture path at d = 1, 3 and 6 and up to the largest mixture the
    C-ABI takes (32 components)."""
    x = wl.random_points(T, d, seed=300 + T, lo=0.15, hi=0.85)
    gmm = tuple(wl.f32_pair(v)[1] for v in wl.gmm_params(K, seed=301 + K, d=d))
    ab = wl.f32_pair(wl.rng(302 + d).standard_normal((T, d)))[1]
    xb, sb, (wb, mb, sgb) = cov.cov_field_svgd_vjp(ctx, dev32(x), 0.15, dev32(ab), gmm=gmm)
    xo, wo, mo, so = orc.svgd_gmm_field_vjp(x, *gmm, 0.15, ab)
    for got, want in ((xb, xo), (mb, mo), (sgb, so), (wb, wo)):
        assert rel_norm(host(got), want) <= TOL
    assert ctx.device_status() == (cov.COV_OK, 0)
