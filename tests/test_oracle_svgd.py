"""Pins of the oracle's reference score and Stein variational field (Eq. 4).

Each check compares the oracle with something other than itself: a library
log-density, a closed form, or a Gaussian-integral mean-field limit.
"""
import json
import os

import numpy as np
import pytest
from scipy.special import logsumexp
from scipy.stats import multivariate_normal

from paper_2511_11514_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _scipy_logq(x, w, mu, sigma):
    terms = [np.log(w[k]) + multivariate_normal(mu[k], sigma[k] ** 2 * np.eye(len(x))).logpdf(x)
             for k in range(len(w))]
    return logsumexp(terms)


def test_gmm_logpdf_matches_scipy(orc):
    w, mu, sigma = wl.gmm_params(4, seed=3)
    for x in wl.random_points(5, 2, seed=4):
        assert orc.gmm_logpdf(x, w, mu, sigma) == pytest.approx(_scipy_logq(x, w, mu, sigma), rel=1e-12)


def test_gmm_score_is_gradient_of_library_logpdf(orc):
    """Central finite difference (step 1e-6) of scipy's mixture log-density."""
    w, mu, sigma = wl.gmm_params(5, seed=11)
    x = wl.random_points(6, 2, seed=12)
    score = orc.gmm_score(x, w, mu, sigma)
    h = 1e-6
    for i in range(len(x)):
        for c in range(2):
            e = np.zeros(2)
            e[c] = h
            fd = (_scipy_logq(x[i] + e, w, mu, sigma) - _scipy_logq(x[i] - e, w, mu, sigma)) / (2 * h)
            assert score[i, c] == pytest.approx(fd, rel=1e-5, abs=1e-4)


def test_gmm_score_single_gaussian_closed_form(orc):
    mu = np.array([[0.4, 0.6]])
    sigma = np.array([0.07])
    x = wl.random_points(8, 2, seed=5)
    score = orc.gmm_score(x, np.array([1.0]), mu, sigma)
    np.testing.assert_allclose(score, -(x - mu) / sigma[0] ** 2, rtol=1e-13)


def test_svgd_single_point_is_score(orc):
    """T = 1: k(x,x) = 1 and its gradient vanishes, so g = score."""
    ex = json.load(open(GOLDEN))["svgd_single_point"]
    x = np.array([ex["x"]])
    score = orc.gmm_score(x, np.array([1.0]), np.array([ex["mu"]]), np.array([ex["sigma"]]))
    g = orc.svgd_field(x, score, h=ex["h"])
    np.testing.assert_allclose(g[0], ex["field"], rtol=1e-13)


def test_svgd_two_points_hand_example(orc):
    """T = 2 with zero score at distance h: worked by hand in the fixture."""
    ex = json.load(open(GOLDEN))["svgd_two_points_zero_score"]
    x = np.array(ex["x"])
    g = orc.svgd_field(x, np.zeros_like(x), h=ex["h"])
    np.testing.assert_allclose(g, ex["field"], rtol=1e-12)


def test_svgd_repulsion_cancels_in_sum(orc):
    """With zero score the kernel-gradient terms are antisymmetric in (i,j),
    so the field sums to zero."""
    x = wl.random_points(17, 2, seed=8)
    g = orc.svgd_field(x, np.zeros_like(x), h=0.2)
    assert np.abs(g.sum(axis=0)).max() < 1e-13 * np.abs(g).max() * len(x)


def _mean_field(xe, mu, sig, m, s, h):
    """Gaussian-integral closed form of E_{x'~N(m, s^2 I)}[k(x', xe) score(x')
    + grad_{x'} k(x', xe)] for q = N(mu, sig^2 I) and the RBF kernel with
    length-scale h (d = 2)."""
    d = len(xe)
    v = h * h + s * s
    Z = (h * h / v) ** (d / 2) * np.exp(-np.sum((xe - m) ** 2) / (2 * v))
    mpost = (h * h * m + s * s * xe) / v            # E[x' k] / E[k]
    return Z * (-(mpost - mu) / sig ** 2 + (xe - mpost) / h ** 2)


def test_svgd_gaussian_mean_field_limit(orc):
    """T = 2^16 particles from N(m, s^2 I), target N(mu, sig^2 I): the field
    at sampled particles matches the Gaussian-integral closed form within
    4 Monte-Carlo standard errors (estimated from 8 independent batches)."""
    mu, sig = np.array([0.3, -0.2]), 0.8
    m, s, h = np.array([0.0, 0.1]), 1.0, 0.7
    T = 1 << 16
    g = wl.rng(21)
    x = m + s * g.standard_normal(size=(T, 2))
    score = -(x - mu) / sig ** 2
    rows = np.arange(8)
    got = orc.svgd_field(x, score, h, rows=rows)
    # batch means -> standard error of the full-T estimate
    B = 8
    bs = T // B
    per_batch = []
    for bi in range(B):
        xb = x[bi * bs:(bi + 1) * bs]
        xb = np.concatenate([x[rows], xb])
        sb = -(xb - mu) / sig ** 2
        per_batch.append(orc.svgd_field(xb, sb, h, rows=rows))
    se = np.std(np.stack(per_batch), axis=0, ddof=1) / np.sqrt(B)
    want = np.stack([_mean_field(x[i], mu, sig, m, s, h) for i in rows])
    assert np.all(np.abs(got - want) <= 4 * se + 1e-12)
    # the pin would catch a flipped repulsive term or a kernel without the 1/2
    flipped = np.stack([_mean_field(x[i], mu, sig, m, s, h) -
                        2 * ((x[i] - (h * h * m + s * s * x[i]) / (h * h + s * s)) / h ** 2) *
                        (h * h / (h * h + s * s)) * np.exp(-np.sum((x[i] - m) ** 2) / (2 * (h * h + s * s)))
                        for i in rows])
    assert np.any(np.abs(got - flipped) > 4 * se)


def test_svgd_row_subset_matches_full(orc):
    x = wl.random_points(33, 2, seed=9)
    sc = orc.gmm_score(x, *wl.gmm_params(3, seed=2))
    full = orc.svgd_field(x, sc, 0.05)
    rows = np.array([0, 5, 32, 7])
    np.testing.assert_array_equal(orc.svgd_field(x, sc, 0.05, rows=rows), full[rows])


# -- reference as a pixel density (bilinear interpolant) ----------------------------
def _centres(n):
    return (np.arange(n) + 0.5) / n


def test_density_value_reproduces_bilinear_functions(orc):
    """The bilinear interpolant is exact for q(x) = (1 + a x0)(1 + b x1)
    between the outermost pixel centres, and equals the pixel values at the
    centres."""
    H, W, a, b = 7, 11, 0.8, -0.4
    cx, cy = _centres(W), _centres(H)
    m = (1 + a * cx)[None, :] * (1 + b * cy)[:, None]
    r = wl.rng(3)
    for _ in range(50):
        x = np.array([r.uniform(cx[0], cx[-1]), r.uniform(cy[0], cy[-1])])
        assert orc.density_value(m, x) == pytest.approx((1 + a * x[0]) * (1 + b * x[1]), rel=1e-13)
    assert orc.density_value(m, np.array([cx[3], cy[5]])) == pytest.approx(m[5, 3], rel=1e-14)


def test_density_score_closed_form(orc):
    H, W, a, b = 9, 6, 0.8, -0.4
    cx, cy = _centres(W), _centres(H)
    m = (1 + a * cx)[None, :] * (1 + b * cy)[:, None]
    r = wl.rng(4)
    x = np.stack([r.uniform(cx[0] + 1e-3, cx[-1] - 1e-3, 40), r.uniform(cy[0] + 1e-3, cy[-1] - 1e-3, 40)], 1)
    sc = orc.density_score(m, x)
    np.testing.assert_allclose(sc[:, 0], a / (1 + a * x[:, 0]), rtol=1e-12)
    np.testing.assert_allclose(sc[:, 1], b / (1 + b * x[:, 1]), rtol=1e-12)


def test_density_score_is_gradient_of_log_value(orc):
    """Central differences of log q (the value pinned above) on a random map,
    away from cell edges; outside the centre range the score is zero."""
    m = wl.density_map(seed=5, n=64)
    r = wl.rng(6)
    x = r.uniform(0.05, 0.95, size=(60, 2))
    sc = orc.density_score(m, x)
    h = 1e-7
    for i in range(60):
        for c in range(2):
            e = np.zeros(2)
            e[c] = h
            fd = (np.log(orc.density_value(m, x[i] + e)) - np.log(orc.density_value(m, x[i] - e))) / (2 * h)
            assert sc[i, c] == pytest.approx(fd, rel=1e-5, abs=1e-6)
    out = np.array([[-0.2, 0.5], [0.5, 1.3], [1.2, -0.1]])
    so = orc.density_score(m, out)
    assert so[0, 0] == 0 and so[1, 1] == 0 and np.all(so[2] == 0)


def test_density_score_of_a_fine_gaussian_map(orc):
    """A 512^2 map of an isotropic Gaussian: the score approaches
    -(x - mu)/sigma^2 (discretisation error O(pixel^2 / sigma^2))."""
    n, mu, sig = 512, np.array([0.45, 0.55]), 0.12
    c = _centres(n)
    m = np.exp(-((c[None, :] - mu[0]) ** 2 + (c[:, None] - mu[1]) ** 2) / (2 * sig ** 2))
    x = wl.rng(7).uniform(0.25, 0.75, size=(200, 2))
    sc = orc.density_score(m, x)
    want = -(x - mu) / sig ** 2
    assert np.linalg.norm(sc - want) <= 2e-2 * np.linalg.norm(want)


# -- reverse mode of the Stein field and of the mixture score -----------------
def _fd(fun, v, step=1e-6):
    """Central differences of the scalar fun at every entry of the array v."""
    g = np.zeros_like(v)
    for idx in np.ndindex(v.shape):
        vp, vm = v.copy(), v.copy()
        vp[idx] += step
        vm[idx] -= step
        g[idx] = (fun(vp) - fun(vm)) / (2 * step)
    return g


@pytest.mark.parametrize("T,d,h", [(7, 2, 0.3), (5, 3, 0.5)])
def test_svgd_vjp_matches_central_differences(orc, T, d, h):
    """<abar, field(x, s)> differentiated by central differences (step 1e-6)
    in every coordinate of x (score held fixed) and of s."""
    rng = wl.rng(20 + T)
    x = rng.uniform(0, 1, size=(T, d))
    s = rng.standard_normal((T, d))
    abar = rng.standard_normal((T, d))
    xbar, sbar = orc.svgd_field_vjp(x, s, h, abar)
    L = lambda xx, ss: float(np.sum(abar * orc.svgd_field(xx, ss, h)))
    np.testing.assert_allclose(xbar, _fd(lambda v: L(v, s), x), rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(sbar, _fd(lambda v: L(x, v), s), rtol=1e-6, atol=1e-8)


def test_svgd_vjp_single_point_and_translation(orc):
    """T = 1: the field is the score itself, so xbar = 0 and sbar = abar.
    With the score held fixed the field depends on x only through
    differences x_i - x_j, so the x-gradient sums to zero over the points."""
    x = np.array([[0.3, 0.6]])
    ab = np.array([[0.7, -1.1]])
    xbar, sbar = orc.svgd_field_vjp(x, np.array([[2.0, -3.0]]), 0.2, ab)
    np.testing.assert_array_equal(xbar, 0.0)
    np.testing.assert_allclose(sbar, ab, rtol=0, atol=0)
    rng = wl.rng(31)
    x = rng.uniform(0, 1, size=(40, 2))
    xbar, _ = orc.svgd_field_vjp(x, rng.standard_normal((40, 2)), 0.1, rng.standard_normal((40, 2)))
    assert np.abs(xbar.sum(0)).max() <= 1e-10 * np.abs(xbar).sum()


def test_gmm_score_vjp_matches_central_differences(orc):
    """sum_i sbar_i . score(x_i) differentiated by central differences in x,
    the raw weights, the means and the standard deviations; the weight
    gradient is orthogonal to the weights (the score depends on w / sum w)."""
    w, mu, sigma = wl.gmm_params(4, seed=41)
    rng = wl.rng(42)
    x = rng.uniform(0.1, 0.9, size=(6, 2))
    sb = rng.standard_normal((6, 2))
    xbar, wbar, mubar, sigbar = orc.gmm_score_vjp(x, w, mu, sigma, sb)
    Ls = lambda xx, ww, mm, ss: float(np.sum(sb * orc.gmm_score(xx, ww, mm, ss)))
    np.testing.assert_allclose(xbar, _fd(lambda v: Ls(v, w, mu, sigma), x), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(wbar, _fd(lambda v: Ls(x, v, mu, sigma), w), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(mubar, _fd(lambda v: Ls(x, w, v, sigma), mu), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(sigbar, _fd(lambda v: Ls(x, w, mu, v), sigma), rtol=1e-6, atol=1e-5)
    assert abs(float(w @ wbar)) <= 1e-10 * float(np.abs(w * wbar).sum())


def test_svgd_with_mixture_score_vjp_is_the_total_derivative(orc):
    """The chained reverse mode (kernel part + score part) against central
    differences of <abar, field(x, score(x))> through both paths."""
    w, mu, sigma = wl.gmm_params(3, seed=51)
    rng = wl.rng(52)
    x = rng.uniform(0.2, 0.8, size=(8, 2))
    abar = rng.standard_normal((8, 2))
    h = 0.15
    xbar, wbar, mubar, sigbar = orc.svgd_gmm_field_vjp(x, w, mu, sigma, h, abar)
    L = lambda xx, ww, mm, ss: float(np.sum(abar * orc.svgd_field(xx, orc.gmm_score(xx, ww, mm, ss), h)))
    np.testing.assert_allclose(xbar, _fd(lambda v: L(v, w, mu, sigma), x), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(mubar, _fd(lambda v: L(x, w, v, sigma), mu), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(sigbar, _fd(lambda v: L(x, w, mu, v), sigma), rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(wbar, _fd(lambda v: L(x, v, mu, sigma), w), rtol=1e-6, atol=1e-6)


def test_svgd_permutation_and_rotation_equivariance(orc):
    """The Stein field of relabelled points is the relabelled field; rotating
    the points and the mixture's means together (isotropic components) rotates
    the score and the field (would catch a swapped i/j or a transposed
    coordinate in either)."""
    w, mu, sigma = wl.gmm_params(4, seed=8, d=2)
    x = wl.random_points(12, 2, seed=9)
    h = 0.1
    a = orc.svgd_field(x, orc.gmm_score(x, w, mu, sigma), h)
    perm = np.random.default_rng(4).permutation(12)
    np.testing.assert_allclose(orc.svgd_field(x[perm], orc.gmm_score(x[perm], w, mu, sigma), h), a[perm],
                               atol=1e-12)
    th = -1.1
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    sc_r = orc.gmm_score(x @ R.T, w, mu @ R.T, sigma)
    np.testing.assert_allclose(sc_r, orc.gmm_score(x, w, mu, sigma) @ R.T, atol=1e-9)
    np.testing.assert_allclose(orc.svgd_field(x @ R.T, sc_r, h), a @ R.T, atol=1e-9)
