"""Autotuner for the tile shape of the all-pairs kernels.

The all-pairs kernel has two knobs (C-ABI options): rows per thread R
(COV_OPT_ROWS_PER_THREAD: 2, 4 or 8 register rows per lane) and the cap on
resident CTAs per SM that the column-split planner fills
(COV_OPT_CTAS_PER_SM).  The best pair depends on the problem shape: small
problems want many short CTAs, large ones more rows per thread.  `tune_*`
times every candidate on the caller's own inputs (for the Sinkhorn field in the
library, cov_autotune_sinkhorn; for the Stein field here through the C-ABI),
with CUDA events, as the per-iteration time (t(n_hi) - t(n_lo)) / (n_hi - n_lo)
so that prep and launch costs cancel; the winner is cached in a JSON file keyed by
GPU name, field kind, d, the power-of-two buckets of T and M and the exponent
path, and applied to the context.

    python -m paper_2511_11514_b300.autotune --workload NAME   # prints the sweep
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

import torch

from . import binding as cov

CANDIDATES = ((2, 8), (4, 8), (8, 8), (4, 6), (2, 6), (8, 4))
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build",
                             "autotune_cache.json")


def _bucket(n: int) -> int:
    return 1 << max(0, (int(n) - 1).bit_length())


def cache_key(kind: str, d: int, T: int, M: int = 0, tc: int = cov.TENSOR_CORES_AUTO) -> str:
    """GPU, field kind, d, the power-of-two buckets of T and M, and the
    exponent path (COV_OPT_TENSOR_CORES) the sweep ran with."""
    name = torch.cuda.get_device_name().replace(" ", "_")
    return f"{name}|{kind}|d{d}|T{_bucket(T)}|M{_bucket(M) if M else 0}|tc{tc}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(ctx: cov.Context, choice: dict) -> None:
    ctx.set_option(cov.OPT_ROWS_PER_THREAD, int(choice["R"]))
    ctx.set_option(cov.OPT_CTAS_PER_SM, int(choice["ctas_per_sm"]))


def _timed(fn, reps: int) -> float:
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def sweep_sinkhorn(ctx, x, y, eps):
    """[(R, ctas_per_sm, us per Sinkhorn iteration)] on these inputs: the
    library's own sweep (cov_autotune_sinkhorn), which also applies the best."""
    _, _, rows = cov.cov_autotune_sinkhorn(ctx, x, y, eps)
    return rows


def sweep_svgd(ctx, x, h, score, candidates=CANDIDATES, reps=5):
    out = []
    for R, cps in candidates:
        apply(ctx, {"R": R, "ctas_per_sm": cps})
        cov.cov_field_svgd(ctx, x, h, score=score)
        out.append((R, cps, 1e3 * _timed(lambda: cov.cov_field_svgd(ctx, x, h, score=score), reps)))
    return out


def tune_sinkhorn(ctx, x, y, eps, cache_path: str = DEFAULT_CACHE, force: bool = False) -> dict:
    """Pick (and apply) the fastest tiling for a Sinkhorn field of this shape.

    The tile shape only shapes the CUDA-core kernel (the tensor-core kernel
    has one shape; the CUDA cores still run the first iteration, the
    gradient passes and any recompute), so the library's sweep runs with
    the tensor cores off whatever the context's setting."""
    key = cache_key("sinkhorn", x.shape[1], x.shape[0], y.shape[0], cov.TENSOR_CORES_OFF)
    cache = load_cache(cache_path)
    if not force and key in cache:
        apply(ctx, cache[key])
        return cache[key]
    res = sweep_sinkhorn(ctx, x, y, eps)
    R, cps, us = min(res, key=lambda r: r[2])
    choice = {"R": R, "ctas_per_sm": cps, "us_per_iteration": us,
              "sweep": [{"R": a, "ctas_per_sm": b, "us": c} for a, b, c in res]}
    cache[key] = choice
    save_cache(cache, cache_path)
    apply(ctx, choice)
    return choice


def tune_svgd(ctx, x, h, score, cache_path: str = DEFAULT_CACHE, force: bool = False) -> dict:
    key = cache_key("svgd", x.shape[1], x.shape[0])
    cache = load_cache(cache_path)
    if not force and key in cache:
        apply(ctx, cache[key])
        return cache[key]
    res = sweep_svgd(ctx, x, h, score)
    R, cps, us = min(res, key=lambda r: r[2])
    choice = {"R": R, "ctas_per_sm": cps, "us_per_field": us,
              "sweep": [{"R": a, "ctas_per_sm": b, "us": c} for a, b, c in res]}
    cache[key] = choice
    save_cache(cache, cache_path)
    apply(ctx, choice)
    return choice


def main():
    from . import workloads as wl
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default=wl.SINKHORN_DOUBLE_T4096.name, choices=sorted(wl.WORKLOADS))
    ap.add_argument("--cache", default=DEFAULT_CACHE)
    args = ap.parse_args()
    w = wl.WORKLOADS[args.workload]
    inst = wl.make_instance(w)
    ctx = cov.Context(0)
    u = torch.as_tensor(inst.u0, dtype=torch.float64, device="cuda")
    s = cov.cov_rollout(ctx, w.model, inst.s0, u, w.dt)
    x = s[1:, :2].float().contiguous()
    if w.field == wl.FIELD_SINKHORN:
        y = torch.as_tensor(inst.y, dtype=torch.float32, device="cuda")
        pairs = 2 * w.T * w.M + w.T * w.T
        choice = tune_sinkhorn(ctx, x, y, w.eps, args.cache, force=True)
        print(f"# {w.name}: pairs per Sinkhorn iteration {pairs:.3e}")
        for r in choice["sweep"]:
            print(f"R={r['R']} ctas_per_sm={r['ctas_per_sm']}: {r['us']:.1f} us/iteration, "
                  f"{pairs / (r['us'] * 1e-6) / 1e12:.2f} Tpair/s")
    else:
        score = cov.cov_gmm_score(ctx, x, inst.gmm)
        choice = tune_svgd(ctx, x, w.h, score, args.cache, force=True)
        for r in choice["sweep"]:
            print(f"R={r['R']} ctas_per_sm={r['ctas_per_sm']}: {r['us']:.1f} us/field")
    print("chosen:", {k: v for k, v in choice.items() if k != "sweep"})
    ctx.close()


if __name__ == "__main__":
    main()
