"""Seeded synthetic inputs for coverage problems (input generation only).

This module holds none of the method's arithmetic: it draws reference
distributions, reference samples and initial trajectories, and names the
benchmark configurations.  It is the one module that both the CUDA path's
tests/benchmark and the CPU oracle's callers use, so that both sides see the
same data.  Everything is float64 from a Philox-4x32-10 generator
(``numpy.random.Philox``); ``f32_pair`` rounds an array to float32 and
returns the float64 image of that rounding, so the GPU (float32) and the
oracle (float64) receive bit-identical values.

The paper names no dataset: references are Gaussian mixtures or a density
map on the unit square (Sec. II-A, "a set of samples" or "a continuous
utility function"), shaped like the benchmarks of Sec. III-A.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
import numpy as np

SINGLE_INT, DOUBLE_INT, UNICYCLE = 0, 1, 2
FIELD_SVGD, FIELD_SINKHORN = 0, 1
MODEL_DIMS = {SINGLE_INT: (2, 2), DOUBLE_INT: (4, 2), UNICYCLE: (3, 2)}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def f32_pair(a):
    """(float32 array, float64 array holding exactly the same values)."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    return a32, a32.astype(np.float64)


# -- reference distributions ----------------------------------------------
def gmm_params(K: int, seed: int, *, mean_lo=0.2, mean_hi=0.8, sig_lo=0.05,
               sig_hi=0.15, dirichlet=True, d=2):
    """Isotropic 2-D mixture: means U[lo,hi]^d, sigma U[sig_lo,sig_hi],
    weights Dirichlet(1) (or uniform)."""
    g = rng(seed)
    mu = g.uniform(mean_lo, mean_hi, size=(K, d))
    sigma = g.uniform(sig_lo, sig_hi, size=K)
    w = g.dirichlet(np.ones(K)) if dirichlet else np.full(K, 1.0 / K)
    return w, mu, sigma


def gmm_samples(w, mu, sigma, M: int, seed: int):
    g = rng(seed)
    comp = g.choice(len(w), size=M, p=np.asarray(w) / np.sum(w))
    return mu[comp] + sigma[comp, None] * g.standard_normal(size=(M, mu.shape[1]))


def density_map(seed: int, n: int = 512, n_gauss: int = 32, floor: float = 0.05):
    """Sum of n_gauss anisotropic Gaussians on an n x n grid over [0,1]^2,
    means U[0,1]^2, axis sigmas U[0.01,0.1], rotation U[0,pi), amplitude
    U[0.5,1]; normalised to mass 1-floor plus a uniform floor.  Returns the
    per-pixel probability map [n, n] (row = y index, column = x index)."""
    g = rng(seed)
    c = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(c, c)
    dens = np.zeros((n, n))
    for _ in range(n_gauss):
        m = g.uniform(0.0, 1.0, size=2)
        s = g.uniform(0.01, 0.1, size=2)
        th = g.uniform(0.0, math.pi)
        amp = g.uniform(0.5, 1.0)
        dx, dy = X - m[0], Y - m[1]
        u = math.cos(th) * dx + math.sin(th) * dy
        v = -math.sin(th) * dx + math.cos(th) * dy
        dens += amp * np.exp(-0.5 * ((u / s[0]) ** 2 + (v / s[1]) ** 2))
    dens *= (1.0 - floor) / dens.sum()
    dens += floor / (n * n)
    return dens


def density_samples(pmap, M: int, seed: int):
    """Pick a pixel by its probability, then jitter uniformly inside it."""
    g = rng(seed)
    n = pmap.shape[0]
    idx = g.choice(n * n, size=M, p=pmap.ravel() / pmap.sum())
    iy, ix = np.divmod(idx, n)
    jit = g.uniform(0.0, 1.0, size=(M, 2))
    return np.stack([(ix + jit[:, 0]) / n, (iy + jit[:, 1]) / n], axis=1)


# -- initial trajectories ---------------------------------------------------
def line_controls_single(T: int, dt: float, seed: int, start=(0.1, 0.1),
                         end=(0.9, 0.9), noise=0.01):
    """Single integrator: controls whose Euler rollout from `start` visits
    the straight line to `end` plus N(0, noise^2) position noise."""
    g = rng(seed)
    t = np.arange(T + 1)[:, None] / T
    pos = np.asarray(start)[None, :] + t * (np.asarray(end) - np.asarray(start))[None, :]
    pos[1:] += noise * g.standard_normal(size=(T, 2))
    return np.asarray(start, dtype=np.float64), (pos[1:] - pos[:-1]) / dt


def double_int_init(T: int, dt: float, start=(0.1, 0.1), span=0.8):
    v0 = span / (T * dt)
    return np.array([start[0], start[1], v0, v0]), np.zeros((T, 2))


def unicycle_init(T: int, dt: float, start=(0.1, 0.1), span=0.8):
    speed = math.hypot(span, span) / (T * dt)
    return np.array([start[0], start[1], math.pi / 4]), np.tile([speed, 0.0], (T, 1))


def coverage_Q(model: int, d: int = 2):
    """Unit weight on the coverage coordinates (the first d state
    components), zero on the others."""
    n, _ = MODEL_DIMS[model]
    Q = np.zeros((n, n))
    Q[np.arange(d), np.arange(d)] = 1.0
    return Q


# -- named workloads ----------------------------------------------------------
@dataclass
class Workload:
    name: str
    model: int
    field: int
    T: int
    dt: float
    n_outer: int
    eta: float
    M: int = 0
    eps: float = 0.0
    n_iter: int = 0
    h: float = 0.0
    R_scale: float = 0.01
    seed: int = 0
    gmm_K: int = 0
    reference: str = "gmm"   # "gmm" or "density"
    extra: dict = field(default_factory=dict)

    @property
    def pairs_per_field(self) -> int:
        """Pair evaluations per field: one (row, column) term of a
        soft-c-transform or SVGD sum."""
        if self.field == FIELD_SVGD:
            return self.T * self.T
        T, M = self.T, self.M
        return self.n_iter * (2 * T * M + T * T) + (T * M + T * T)


SVGD_SINGLE_T256 = Workload(
    name="svgd_single_integrator_T256", model=SINGLE_INT, field=FIELD_SVGD,
    T=256, dt=0.1, n_outer=100, eta=1e-3, h=0.05, gmm_K=3)

SINKHORN_DOUBLE_T4096 = Workload(
    name="sinkhorn_double_integrator_T4096_M16384", model=DOUBLE_INT,
    field=FIELD_SINKHORN, T=4096, dt=0.05, n_outer=200, eta=0.5, M=16384,
    eps=0.005, n_iter=50, gmm_K=8)

SINKHORN_UNICYCLE_T65536 = Workload(
    name="sinkhorn_unicycle_T65536_M262144", model=UNICYCLE,
    field=FIELD_SINKHORN, T=65536, dt=0.01, n_outer=10, eta=0.5, M=262144,
    eps=0.002, n_iter=100, reference="density")

# Differentiation: gradient of the coverage loss (Sinkhorn divergence of the
# final trajectory to a held-out 4-component mixture, M = 8192 samples drawn
# with seed 1, uniform weights) through 20 outer iterations with respect to
# the reference mixture's means, log-sigmas and weight logits (samples by
# reparameterisation, M/4 per component) and the initial state.
ADJOINT_DOUBLE_T2048 = Workload(
    name="adjoint_double_integrator_T2048_M8192_K20", model=DOUBLE_INT,
    field=FIELD_SINKHORN, T=2048, dt=0.05, n_outer=20, eta=0.5, M=8192,
    eps=0.005, n_iter=50, gmm_K=4,
    extra={"loss_M": 8192, "loss_seed": 1, "loss_eps": 0.005, "loss_iters": 100})

WORKLOADS = {w.name: w for w in (SVGD_SINGLE_T256, SINKHORN_DOUBLE_T4096,
                                 SINKHORN_UNICYCLE_T65536, ADJOINT_DOUBLE_T2048)}


@dataclass
class Instance:
    """Concrete float64 inputs of one workload (already float32-exact where
    the GPU consumes them as float32)."""
    wl: Workload
    s0: np.ndarray
    u0: np.ndarray
    Q: np.ndarray
    R: np.ndarray
    y: np.ndarray | None = None       # [M,2] float32-exact
    b: np.ndarray | None = None       # [M] float32-exact, or None (uniform)
    gmm: tuple | None = None          # (w, mu, sigma) float64


def make_instance(wl: Workload, *, T: int | None = None, M: int | None = None,
                  seed: int | None = None) -> Instance:
    """Build the inputs of `wl`, optionally at a reduced size (T, M)."""
    T = wl.T if T is None else T
    M = wl.M if M is None else M
    seed = wl.seed if seed is None else seed
    if wl.model == SINGLE_INT:
        s0, u0 = line_controls_single(T, wl.dt, seed)
    elif wl.model == DOUBLE_INT:
        s0, u0 = double_int_init(T, wl.dt)
    else:
        s0, u0 = unicycle_init(T, wl.dt)
    n, m = MODEL_DIMS[wl.model]
    Q = np.eye(n) if wl.model == SINGLE_INT else coverage_Q(wl.model)
    R = wl.R_scale * np.eye(m)
    inst = Instance(wl=wl, s0=s0, u0=u0, Q=Q, R=R)
    if wl.reference == "gmm":
        dirichlet = wl.field == FIELD_SVGD
        w, mu, sigma = gmm_params(wl.gmm_K, seed, dirichlet=dirichlet)
        inst.gmm = (w, mu, sigma)
        if wl.field == FIELD_SINKHORN:
            inst.y = f32_pair(gmm_samples(w, mu, sigma, M, seed + 1000))[1]
    else:
        pmap = density_map(seed)
        inst.y = f32_pair(density_samples(pmap, M, seed + 1000))[1]
    return inst


def random_points(n: int, d: int, seed: int, lo=0.0, hi=1.0):
    """Uniform points in [lo,hi]^d, float32-exact."""
    return f32_pair(rng(seed).uniform(lo, hi, size=(n, d)))[1]


def random_weights(n: int, seed: int):
    """Positive weights summing to 1 up to float32 rounding (float32-exact,
    so both sides see the same numbers; neither side renormalises)."""
    w = rng(seed).uniform(0.5, 1.5, size=n)
    w32 = (w / w.sum()).astype(np.float32)
    return w32.astype(np.float64)


# -- batched workload: many independent problems of uneven size ---------------
def make_batch(n: int, seed: int = 0, T_range=(128, 4096), M_range=(512, 16384), K_range=(2, 16)):
    """n double-integrator coverage problems; T ~ U{T_range}, M ~ U{M_range},
    each with its own 2-16 component mixture (seed = problem index); even
    indices use the Stein field, odd ones the Sinkhorn field (eps = 0.005,
    50 iterations).  Returns a list of Instance."""
    g = rng(seed)
    out = []
    for p in range(n):
        T = int(g.integers(T_range[0], T_range[1] + 1))
        M = int(g.integers(M_range[0], M_range[1] + 1))
        K = int(g.integers(K_range[0], K_range[1] + 1))
        svgd = p % 2 == 0
        w = Workload(name=f"batch_{p}", model=DOUBLE_INT, field=FIELD_SVGD if svgd else FIELD_SINKHORN, T=T,
                     dt=0.05, n_outer=100, eta=1e-3 if svgd else 0.5, M=0 if svgd else M, eps=0.0 if svgd else 0.005,
                     n_iter=0 if svgd else 50, h=0.05 if svgd else 0.0, gmm_K=K, seed=p)
        s0, u0 = double_int_init(T, w.dt)
        wts, mu, sigma = gmm_params(K, seed=p, dirichlet=True)
        inst = Instance(wl=w, s0=s0, u0=u0, Q=coverage_Q(DOUBLE_INT), R=w.R_scale * np.eye(2),
                        gmm=tuple(f32_pair(v)[1] for v in (wts, mu, sigma)))
        if not svgd:
            inst.y = f32_pair(gmm_samples(wts, mu, sigma, M, seed=p + 100000))[1]
        out.append(inst)
    return out
