#!/usr/bin/env python
"""Benchmark of the coverage hot path: one outer iteration (a "step") of the
Sinkhorn coverage solve on the large unicycle workload -- T = 65536
trajectory samples, M = 262144 reference samples from a 512 x 512 density
map, eps = 0.002, 100 log-domain Sinkhorn iterations per field, FP32 field +
FP64 LQR/rollout -- through the C-ABI (cov_solve_continue).  The
double-integrator workload (T = 4096, M = 16384, 50 iterations) is measured
beside it as a secondary figure.

Prints ONE JSON line (rank 0).  `value` is pair evaluations per second over
all ranks (one independent coverage problem per rank, weak scaling); one
pair evaluation is one (row, column) term of a soft-c-transform, so a field
costs n_iter (2TM + T^2) + (TM + T^2) of them.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
      [--workload NAME]

`--impl reference` times the FP64 CPU oracle on the host cores (bounded
row samples of the same workload); it is the reference arm.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2511_11514_b300 import workloads as wl  # noqa: E402

METRIC = "pair-evals/s & ms per coverage solve (field % of FP32/SFU roofline) vs FP64 oracle"
UNIT = "pair-evals/s"
DEFAULT_WORKLOAD = wl.SINKHORN_UNICYCLE_T65536.name
L2_FLUSH_BYTES = 256 << 20
# Algorithmic FP32-pipe instructions per Sinkhorn pair evaluation (base-2,
# prescaled, column term folded) in the fixed-offset form the iteration runs
# in from its second step: 2 FMA for the d = 2 inner product, the offset
# subtraction and the accumulation; one exponential (MUFU ex2).  With 128
# FP32 lanes and 32 ex2 per SM and clock both pipes bound at 32 pairs/clk/SM.
FP32_OPS_PER_PAIR = 4
SM_COUNT_NOMINAL = 148
SM_MAX_MHZ_NOMINAL = 2032.0
FP32_LANES_PER_SM_CLK = 128
# DRAM bytes (read + write) per launch of pairs_kernel at the double-
# integrator workload from one ncu capture of the current kernel (fixed-
# offset form): 393 KB (g + p launch) and 290 KB (f launch), no writes.
PAIRS_TRAFFIC_BYTES = 341504
# The same for lse_tc_kernel at T = 65536, M = 262144 (the default path at
# that size): 9.47 MB (g + p launch) and 13.50 MB (f launch), no writes.
TC_LARGE_TRAFFIC_BYTES = 11485824


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(wl.WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-tune", action="store_true", help="skip the tile-shape autotuner")
    ap.add_argument("--batched", type=int, default=0,
                    help="time cov_solve_batched on this many uneven problems (and the same problems one by one)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary measurement of the other Sinkhorn workload")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the differentiation workload: forward and backward through 20 outer iterations")
    ap.add_argument("--variants", action="store_true",
                    help="measure the Sinkhorn variants at eps = 0.002: iterations to a field accuracy, "
                         "cold vs eps-scaled vs warm-started")
    ap.add_argument("--horizon-sweep", action="store_true",
                    help="solve time against the horizon T in the shape of the paper's timing study: Stein field "
                         "(unicycle, T = 100..10000) and Sinkhorn field (double integrator, M = T, T = 100..2500), "
                         "on the GPU and on the FP64 oracle (context, not the headline)")
    ap.add_argument("--lqr-sweep", default="",
                    help="comma-separated horizons: time the LQR step (cov_lqr_track: parallel-in-time Riccati + "
                         "the two affine scans) on the unicycle linearisation at each T (context)")
    ap.add_argument("--batch-share", type=int, default=0,
                    help="--batched: percent of the GPU each problem's all-pairs launches plan for "
                         "(COV_OPT_BATCH_SHARE; 0 keeps the library default)")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="form the fixed-offset updates' exponents on the tensor cores (COV_OPT_TENSOR_CORES)")
    ap.add_argument("--field-profile", default="",
                    help="T,M: run only Sinkhorn field evaluations (--steps of them, 8 iterations each, on the "
                         "default exponent path) of the workload's trajectory and reference at this size, with "
                         "the profiler range around them: a short target for ncu")
    ap.add_argument("--adjoint-outer", type=int, default=0,
                    help="outer iterations of --adjoint (default: the workload's 20; fewer only to keep a "
                         "profiler's launch list short)")
    return ap.parse_args()


def count_library_launches(step) -> int:
    """Kernels of libcov (names in namespace cov::) that one call of `step`
    launches, counted from CUDA activity records of one untimed run."""
    import torch
    from torch.profiler import ProfilerActivity, profile
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        step()
        torch.cuda.synchronize()
    return int(sum(e.count for e in prof.key_averages() if "cov::" in e.key))


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(value, world, device="cpu"):
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, pairs_per_step, steps, max_total_ms):
    """Whole-job pair evaluations per second: every rank solves its own
    problem of the same size (weak scaling), timed by the slowest rank."""
    return world * pairs_per_step * steps / (max_total_ms * 1e-3)


def assign_problems(costs, world):
    """Independent problems to ranks by cost (longest first, each to the rank
    with the least work so far, ties to the lower rank): a deterministic
    partition every rank computes identically, so no collective is needed
    to agree on it.  Returns one list of problem indices per rank, each in
    increasing order."""
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for p in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(p)
        load[r] += costs[p]
    return [sorted(o) for o in out]


# -- clocks sampled during the timed region ------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.index = vis.split(",")[local_rank] if vis else str(local_rank)
        self.proc = None

    def start(self):
        self.out = tempfile.TemporaryFile(mode="w+")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        sm, mx, pw, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.out.read().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
                pw.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "sm_mhz_min": min(sm),
                "power_w_max": max(pw), "samples": len(sm), "reasons": sorted(reasons)}


# -- CPU oracle timing (reference arm and cpu_baseline) ---------------------------
def oracle_sample(inst, rows, seed=0, iters=1):
    """A bounded sample of the workload on the oracle: `iters` chained
    Sinkhorn iterations from the initial trajectory, each over `rows` rows
    of every update (g, f, p; all rows once `rows` reaches the set size).
    Returns (pairs, seconds)."""
    import oracle as orc
    w = inst.wl
    s = orc.rollout(w.model, inst.s0, inst.u0, w.dt)
    x = wl.f32_pair(s[1:, :2])[1]
    y = inst.y
    T, M = len(x), len(y)
    r = wl.rng(seed)
    ry = r.choice(M, size=min(rows, M), replace=False)
    rx = r.choice(T, size=min(rows, T), replace=False)
    f, g, p = np.zeros(T), np.zeros(M), np.zeros(T)
    t0 = time.perf_counter()
    for _ in range(iters):
        g[ry] = orc.sinkhorn_g_update(x, y, w.eps, f, rows=ry)
        f[rx] = orc.sinkhorn_f_update(x, y, None, w.eps, g, rows=rx)
        p[rx] = orc.sinkhorn_p_update(x, w.eps, p, rows=rx)
    dt = time.perf_counter() - t0
    return iters * (len(ry) * T + len(rx) * M + len(rx) * T), dt


def calibrate(inst, seconds):
    """(rows, iterations) of a sample that takes about `seconds`."""
    import oracle as orc
    orc.set_threads(os.cpu_count() or 1)
    pairs, dt = oracle_sample(inst, 64)
    rate = pairs / max(dt, 1e-9)
    per_row = pairs / 64
    rows = max(64, int(seconds * rate / per_row))
    T, M = inst.wl.T, inst.wl.M
    if rows <= min(T, M):
        return rows, 1
    # full iterations: the small sample underrates the cores, and the first
    # full one (thread start-up, first touch of its buffers) overrates the time
    oracle_sample(inst, max(T, M))
    _, dt_two = oracle_sample(inst, max(T, M), iters=2)
    return max(T, M), max(1, int(round(seconds / max(dt_two / 2, 1e-9))))


def host_cpu():
    """The host's processor model (/proc/cpuinfo) and hardware thread count,
    reported beside every oracle timing."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "hardware_threads": os.cpu_count() or 1}


def cpu_baseline(inst, seconds, single_thread_seconds=None):
    """The FP64 oracle's pair-evaluation rate on a bounded sample of the
    workload (rows of each Sinkhorn update, or whole iterations when they
    fit), on all host cores and, for about a third of the time, on one
    thread.  The rate is per pair evaluation, so it extrapolates to the whole
    workload (the oracle's work per pair does not depend on the sample)."""
    import oracle as orc
    cores = os.cpu_count() or 1
    orc.set_threads(cores)
    rows, iters = calibrate(inst, seconds)
    pairs, dt = oracle_sample(inst, rows, seed=1, iters=iters)
    # the host cores' speed varies between the calibration and the sample
    # (shared host): top the sample up once if it fell well short
    if dt < 0.8 * seconds:
        more = max(1, int(round(iters * (seconds - dt) / max(dt, 1e-9))))
        p2, d2 = oracle_sample(inst, rows, seed=2, iters=more)
        pairs, dt, iters = pairs + p2, dt + d2, iters + more
    T, M = inst.wl.T, inst.wl.M
    what = (f"{rows} rows of each Sinkhorn update" if iters == 1 else
            f"{iters} full Sinkhorn iterations (g over T={T}, f over M={M}, p over T)")
    w = inst.wl
    rate = pairs / dt
    out = {"value": rate, "unit": UNIT, "cores": orc.get_threads(), "kind": "oracle", **host_cpu(),
           "sample": f"FP64 oracle: {what} of the workload from its initial trajectory, {pairs:.3e} pair "
                     f"evaluations in {dt:.1f} s, {orc.get_threads()} threads",
           "extrapolated": {"ms_per_step": w.pairs_per_field / rate * 1e3,
                            "ms_per_coverage_solve": w.n_outer * w.pairs_per_field / rate * 1e3,
                            "how": "the sample's pair rate applied to the whole step / solve"}}
    st = seconds / 3 if single_thread_seconds is None else single_thread_seconds
    if st > 0:
        orc.set_threads(1)
        try:
            p1, d1 = oracle_sample(inst, 16)
            r1 = max(16, min(min(T, M), int(16 * st / max(d1, 1e-9))))
            p1, d1 = oracle_sample(inst, r1, seed=3)
        finally:
            orc.set_threads(cores)
        out["single_thread"] = {"value": p1 / d1, "unit": UNIT, "cores": 1,
                                "sample": f"{r1} rows of each Sinkhorn update, {p1:.3e} pair evaluations in "
                                          f"{d1:.1f} s, 1 thread",
                                "ms_per_step_extrapolated": w.pairs_per_field / (p1 / d1) * 1e3}
    return out


def workload_config(w, extra=None):
    cfg = {"workload": w.name, "T": w.T, "M": w.M, "d": 2, "eps": w.eps, "n_iter": w.n_iter,
           "model": {0: "single_integrator", 1: "double_integrator", 2: "unicycle"}[w.model],
           "reference": "8-component Gaussian mixture" if w.reference == "gmm" else "512x512 density map",
           "pairs_per_step": w.pairs_per_field, "outer_iterations_per_solve": w.n_outer,
           "precision": "f32 field (MUFU ex2.approx), f64 LQR and rollout"}
    if extra:
        cfg.update(extra)
    return cfg


def run_reference(args):
    rank, local_rank, world = dist_env()
    if rank != 0:
        return 0
    import oracle as orc
    orc.build()
    w = wl.WORKLOADS[args.workload]
    inst = wl.make_instance(w)
    orc.set_threads(os.cpu_count() or 1)
    # each step a bounded sample, sized so that the whole run stays within
    # about two and a half minutes whatever --steps/--warmup are
    per_step_s = min(3.0, max(0.05, 150.0 / max(1, args.steps + args.warmup)))
    rows, iters = calibrate(inst, per_step_s)
    for k in range(args.warmup):
        oracle_sample(inst, rows, seed=100 + k, iters=iters)
    tot_pairs, tot_s = 0, 0.0
    for k in range(args.steps):
        p, dt = oracle_sample(inst, rows, seed=k, iters=iters)
        tot_pairs += p
        tot_s += dt
    value = tot_pairs / tot_s
    sample = (f"FP64 oracle, per step {iters} chained Sinkhorn iteration(s) over {rows} rows of each update "
              f"(g, f, p) of the workload, {orc.get_threads()} threads")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Philox)",
            "impl": "reference",
            "config": workload_config(w, {"sample_rows_per_update": rows, "sample_iterations": iters,
                                          "precision": "f64 throughout (the oracle)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.get_threads(), "kind": "oracle", **host_cpu(),
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -- our arm ------------------------------------------------------------------------
def sinkhorn_iteration_ms(cov, ctx, x, y, eps, n_lo, n_hi, reps, flush, stream):
    """Time of one fixed-offset Sinkhorn iteration (two all-pairs launches:
    g + p, then f) on the context's current exponent path, with CUDA events
    on the launching stream: the median over `reps` of
    (t(n_hi iterations) - t(n_lo)) / (n_hi - n_lo), so that the prep, the
    first (running-maximum) iteration and the finish cancel."""
    import torch

    def field_ms(n):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cov.cov_field_sinkhorn(ctx, x, y, eps, n, field=False)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    cov.cov_field_sinkhorn(ctx, x, y, eps, 1, field=False)
    return statistics.median((field_ms(n_hi) - field_ms(n_lo)) / (n_hi - n_lo) for _ in range(reps))


def time_steps(cov, ctx, prob, u, s, steps, flush, stream):
    """Per-step CUDA-event times (ms) of `steps` outer iterations through
    cov_solve_continue, the L2 flushed between steps outside the events."""
    import torch
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev0[k].record(stream)
        cov.cov_solve_continue(ctx, prob, 1, u, s)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(ev0, ev1)]


def sinkhorn_setup(cov, ctx, w, dev, seed, tune):
    """Instance, device inputs, problem, controls and initial rollout of a
    Sinkhorn workload; the autotuned tile shape applied to ctx when `tune`."""
    import torch
    inst = wl.make_instance(w, seed=seed)
    y = torch.as_tensor(inst.y, dtype=torch.float32, device=dev).contiguous()
    prob = cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, y=y, eps=w.eps,
                            n_iter=w.n_iter)
    u = torch.as_tensor(inst.u0, dtype=torch.float64, device=dev).contiguous()
    s = cov.cov_solve(ctx, prob, 0, u)  # trajectory of the initial controls
    tiling = {"R": ctx.option(cov.OPT_ROWS_PER_THREAD, 4), "ctas_per_sm": ctx.option(cov.OPT_CTAS_PER_SM, 8),
              "source": "default"}
    if tune:
        from paper_2511_11514_b300 import autotune
        ch = autotune.tune_sinkhorn(ctx, s[1:, :2].float().contiguous(), y, w.eps)
        tiling = {"R": ch["R"], "ctas_per_sm": ch["ctas_per_sm"], "source": "autotune (before the timed region)"}
    return inst, y, prob, u, s, tiling


def uses_tensor_cores(w, forced):
    """The exponent path the default setting takes: the tensor cores when
    both launches of a Sinkhorn iteration hold at least 2^30 pairs."""
    return forced or min(w.M * w.T + w.T * w.T, w.T * w.M) >= 2 ** 30


def roofline_peaks(probe, num_sms):
    """ALU roofline in pair evaluations/s at the maximum SM clock on two
    bases: (a) the log-sum-exp with a running maximum, 5 FP32-pipe operations
    and one exponential per pair, min(128 FP32 lanes / 5, MUFU ex2 width) per
    SM and clock; (b) the fixed-row-offset form the iterations 2.. run in,
    4 FP32 operations and one exponential, min(128 / 4, MUFU width).  The
    MUFU ex2 width per SM and clock is read from the probe (rounded to a
    power of two)."""
    clk = probe["sm_clock_mhz"] * 1e6
    ex2_per_sm_clk = probe["ex2_lane_ops_s"] / (num_sms * clk)
    width = 2 ** round(np.log2(max(ex2_per_sm_clk, 1.0)))
    base = SM_COUNT_NOMINAL * SM_MAX_MHZ_NOMINAL * 1e6
    mufu = base * width
    fp32_5 = base * FP32_LANES_PER_SM_CLK / 5
    fp32_4 = base * FP32_LANES_PER_SM_CLK / FP32_OPS_PER_PAIR
    return min(fp32_5, mufu), min(fp32_4, mufu), {
        "mufu_ex2_per_sm_clk": width, "mufu_pairs_s": mufu, "fp32_pairs_s_5_ops": fp32_5,
        "fp32_pairs_s_4_ops": fp32_4, "probe_ex2_per_sm_clk_measured": ex2_per_sm_clk}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2511_11514_b300 import binding as cov

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    w = wl.WORKLOADS[args.workload]
    if w.field != wl.FIELD_SINKHORN:
        return run_svgd(args, w, rank, local_rank, world)
    ctx = cov.Context(local_rank)
    if args.tensor_cores:
        ctx.set_option(cov.OPT_TENSOR_CORES, cov.TENSOR_CORES_ON)
    dev = torch.device("cuda", local_rank)
    inst, y, prob, u, s, tiling = sinkhorn_setup(cov, ctx, w, dev, w.seed + rank, not args.no_tune)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        cov.cov_solve_continue(ctx, prob, 1, u, s)
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    clocks = Clocks(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.2)
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees the timed steps only
    t0 = time.perf_counter()
    step_ms = time_steps(cov, ctx, prob, u, s, args.steps, flush, stream)
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    st, flags = ctx.device_status()
    if st != cov.COV_OK:
        raise SystemExit(f"device status {cov.status_string(st)} flags {flags}")
    pairs_step = w.pairs_per_field
    value = job_value(world, pairs_step, args.steps, total_ms)
    ms_per_step = total_ms / args.steps
    tc_path = uses_tensor_cores(w, args.tensor_cores)

    # ---- roofline of the dominant kernel: the Sinkhorn iteration's two
    # all-pairs launches on the path the default setting takes, right after
    # the timed region on the same inputs and stream ----------------------------
    large = w.T * w.M >= 1 << 30
    n_lo, n_hi, reps = (3, 5, 3) if large else (4, 24, 5)
    x = s[1:, :2].float().contiguous()
    t_iter_ms = sinkhorn_iteration_ms(cov, ctx, x, y, w.eps, n_lo, n_hi, reps, flush, stream)
    other_mode = cov.TENSOR_CORES_OFF if tc_path else cov.TENSOR_CORES_ON
    ctx.set_option(cov.OPT_TENSOR_CORES, other_mode)
    t_other_ms = sinkhorn_iteration_ms(cov, ctx, x, y, w.eps, n_lo, n_hi, reps, flush, stream)
    ctx.set_option(cov.OPT_TENSOR_CORES, cov.TENSOR_CORES_ON if args.tensor_cores else cov.TENSOR_CORES_AUTO)
    if not args.no_tune:
        from paper_2511_11514_b300 import autotune
        autotune.apply(ctx, {"R": tiling["R"], "ctas_per_sm": tiling["ctas_per_sm"]})
    pairs_iter = 2 * w.T * w.M + w.T * w.T
    achieved = pairs_iter / (t_iter_ms * 1e-3)
    probe = cov.cov_probe_peaks(ctx, 4096)
    peak, peak_fixed, peak_info = roofline_peaks(probe, torch.cuda.get_device_properties(dev).multi_processor_count)
    traffic = None
    if w.name == wl.SINKHORN_DOUBLE_T4096.name and not tc_path:
        traffic = PAIRS_TRAFFIC_BYTES
    elif w.name == wl.SINKHORN_UNICYCLE_T65536.name and tc_path:
        traffic = TC_LARGE_TRAFFIC_BYTES

    # ---- the LQR step of this workload (linearisation at the current
    # trajectory, parallel-in-time Riccati + the two affine scans) ---------------
    A, B = cov.cov_linearize(ctx, w.model, s, u, w.dt)
    abar = torch.zeros((w.T, A.shape[1]), dtype=torch.float64, device=dev)
    abar[:, :2] = 0.05
    cov.cov_lqr_track(ctx, A, B, inst.Q, inst.R, abar)
    la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    la.record(stream)
    for _ in range(5):
        cov.cov_lqr_track(ctx, A, B, inst.Q, inst.R, abar)
    lb.record(stream)
    torch.cuda.synchronize()
    lqr_ms = la.elapsed_time(lb) / 5
    del A, B, abar

    # ---- one whole coverage solve from the initial controls on a context of
    # its own (workspace reserved before the clock starts): initial rollout,
    # Riccati gains of a time-invariant model, graph capture, every outer
    # iteration -------------------------------------------------------------------
    solve = None
    if rank == 0:
        c2 = cov.Context(local_rank)
        n, m = wl.MODEL_DIMS[w.model]
        c2.reserve_for(w.T, w.M, 2, n, m)
        if not args.no_tune:
            from paper_2511_11514_b300 import autotune
            autotune.apply(c2, {"R": tiling["R"], "ctas_per_sm": tiling["ctas_per_sm"]})
        if args.tensor_cores:
            c2.set_option(cov.OPT_TENSOR_CORES, cov.TENSOR_CORES_ON)
        u2 = torch.as_tensor(inst.u0, dtype=torch.float64, device=dev).contiguous()
        s2 = torch.empty_like(s)
        torch.cuda.synchronize()
        sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        sa.record(stream)
        cov.cov_solve(c2, prob, w.n_outer, u2, s2)
        sb.record(stream)
        torch.cuda.synchronize()
        solve = {"outer_iterations": w.n_outer, "ms": sa.elapsed_time(sb),
                 "host_wall_ms": (time.perf_counter() - h0) * 1e3,
                 "how": "cov_solve from the initial controls on a fresh context (workspace reserved beforehand): "
                        "initial rollout, graph capture, every outer iteration; CUDA events on the stream"}
        st2, fl2 = c2.device_status()
        c2.close()
        if st2 != cov.COV_OK:
            raise SystemExit(f"device status {cov.status_string(st2)} flags {fl2}")

    # ---- end to end through the C-ABI with host buffers ---------------------------
    u_h = torch.as_tensor(inst.u0, dtype=torch.float64).pin_memory()
    y_h = torch.as_tensor(inst.y, dtype=torch.float32).pin_memory()
    u_out = torch.empty_like(u_h).pin_memory()
    s_out = torch.empty((w.T + 1, s.shape[1]), dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.e2e_steps, int(8000.0 / max(ms_per_step, 1e-3))))
    e_ms = []
    for k in range(e2e_steps + 2):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        u.copy_(u_h, non_blocking=True)
        y.copy_(y_h, non_blocking=True)
        cov.cov_solve(ctx, prob, 1, u, s)
        u_out.copy_(u, non_blocking=True)
        s_out.copy_(s, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if k >= 2:
            e_ms.append(a.elapsed_time(b))
    e2e_ms = statistics.mean(e_ms)
    h2d = u_h.numel() * 8 + y_h.numel() * 4
    d2h = u_out.numel() * 8 + s_out.numel() * 8

    launches_per_step = count_library_launches(lambda: cov.cov_solve_continue(ctx, prob, 1, u, s))

    # ---- the other Sinkhorn workload, as a secondary figure (rank 0) --------------
    secondary = None
    if rank == 0 and not args.no_secondary:
        w2 = (wl.SINKHORN_DOUBLE_T4096 if w.name == wl.SINKHORN_UNICYCLE_T65536.name
              else wl.SINKHORN_UNICYCLE_T65536)
        c3 = cov.Context(local_rank)
        if args.tensor_cores:
            c3.set_option(cov.OPT_TENSOR_CORES, cov.TENSOR_CORES_ON)
        inst2, y2, prob2, u3, s3, tiling2 = sinkhorn_setup(cov, c3, w2, dev, w2.seed, not args.no_tune)
        for _ in range(3):
            cov.cov_solve_continue(c3, prob2, 1, u3, s3)
        k2 = 20 if w2.T * w2.M < 1 << 30 else 3
        ms2 = time_steps(cov, c3, prob2, u3, s3, k2, flush, stream)
        large2 = w2.T * w2.M >= 1 << 30
        lo2, hi2, reps2 = (3, 5, 3) if large2 else (4, 24, 5)
        x3 = s3[1:, :2].float().contiguous()
        ti2 = sinkhorn_iteration_ms(cov, c3, x3, y2, w2.eps, lo2, hi2, reps2, flush, stream)
        ach2 = (2 * w2.T * w2.M + w2.T * w2.T) / (ti2 * 1e-3)
        tc2 = uses_tensor_cores(w2, args.tensor_cores)
        secondary = {"workload": w2.name, "T": w2.T, "M": w2.M, "eps": w2.eps, "n_iter": w2.n_iter,
                     "steps": k2, "ms_per_step": statistics.mean(ms2),
                     "value": w2.pairs_per_field / (statistics.mean(ms2) * 1e-3), "unit": UNIT,
                     "tiling": tiling2,
                     "roofline": {"achieved": ach2 / 1e9, "unit": "Gpair/s", "frac": ach2 / peak,
                                  "frac_fixed_offset_basis": ach2 / peak_fixed,
                                  "ms_per_sinkhorn_iteration": ti2,
                                  "kernel": "lse_tc_kernel" if tc2 else "pairs_kernel"}}
        st3, fl3 = c3.device_status()
        c3.close()
        if st3 != cov.COV_OK:
            raise SystemExit(f"device status {cov.status_string(st3)} flags {fl3}")

    if rank == 0:
        kernel = ("lse_tc_kernel (tcgen05 exponents) for the fixed-offset iterations, pairs_kernel for the rest"
                  if tc_path else "pairs_kernel (Sinkhorn g/f/p soft-c-transform)")
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Philox; " + ("density-map samples)" if w.reference == "density" else
                                                   "Gaussian-mixture samples)"),
            "config": workload_config(w, {
                "parallelism": f"{world} independent problems (one per GPU)" if world > 1 else "single GPU",
                "l2": "flushed between steps (256 MiB write outside the per-step CUDA events)",
                "ms_per_coverage_solve": solve["ms"] if solve else None,
                "coverage_solve": solve,
                "lqr_track_ms": lqr_ms,
                "tiling": tiling,
                "exponents": "tensor cores (tcgen05 kind::tf32)" if tc_path else "CUDA cores (FP32 FMA)",
                "wall_s_timed_region": wall}),
            "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "frac_fixed_offset_basis": achieved / peak_fixed,
                         "peak_fixed_offset_basis": peak_fixed / 1e9,
                         "ms_per_sinkhorn_iteration": t_iter_ms,
                         "other_exponent_path": {
                             "path": "CUDA cores (pairs_kernel)" if tc_path else "tensor cores (lse_tc_kernel)",
                             "ms_per_sinkhorn_iteration": t_other_ms,
                             "frac": pairs_iter / (t_other_ms * 1e-3) / peak},
                         "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum per launch of the "
                                         "fixed-offset kernel at this workload, one ncu capture of the current "
                                         "kernel (null where none was taken)",
                         "kernel": kernel + ", per Sinkhorn iteration of 2 launches (g + p, f), "
                                   f"(t({n_hi} iterations) - t({n_lo})) / {n_hi - n_lo}, median of {reps}",
                         "peak_basis": "148 SMs x 2032 MHz x min(MUFU ex2 width, 128 FP32 lanes / 5 operations "
                                       "per pair of the log-sum-exp with a running maximum); "
                                       "peak_fixed_offset_basis: / 4 operations of the fixed-offset form",
                         "peak_detail": peak_info, "probe": probe},
            "secondary": secondary,
            "clocks": clk,
            "e2e": {"value": pairs_step / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": e2e_steps},
            "gpu_launches": launches_per_step * args.steps,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(inst, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_field_profile(args):
    """Sinkhorn field evaluations alone (8 iterations each) at a chosen size
    of the workload (its initial trajectory's positions, its reference
    generator), bracketed by the profiler range: with ncu's
    --profile-from-start off only these launches are seen."""
    import torch

    from paper_2511_11514_b300 import binding as cov

    w = wl.WORKLOADS[args.workload]
    T, M = (int(v) for v in args.field_profile.split(","))
    torch.cuda.set_device(0)
    inst = wl.make_instance(w, T=T, M=M)
    ctx = cov.Context(0)
    dev = torch.device("cuda", 0)
    u = torch.as_tensor(inst.u0, dtype=torch.float64, device=dev)
    x = cov.cov_rollout(ctx, w.model, inst.s0, u, w.dt)[1:, :2].float().contiguous()
    y = torch.as_tensor(inst.y, dtype=torch.float32, device=dev).contiguous()
    cov.cov_field_sinkhorn(ctx, x, y, w.eps, 8, field=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    a.record()
    for _ in range(args.steps):
        cov.cov_field_sinkhorn(ctx, x, y, w.eps, 8, field=False)
    b.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    st, flags = ctx.device_status()
    ctx.close()
    if st != cov.COV_OK:
        raise SystemExit(f"device status {cov.status_string(st)} flags {flags}")
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"field_profile": {"workload": w.name, "T": T, "M": M, "eps": w.eps, "iterations": 8,
                                        "ms_per_field": ms, "evaluations": args.steps,
                                        "tensor_cores": uses_tensor_cores(dataclasses.replace(w, T=T, M=M), False)}}),
          flush=True)
    return 0


def run_svgd(args, w, rank, local_rank, world):
    """The Stein-field workload (latency-bound: T^2 pair evaluations per
    field).  A step is one outer iteration through `cov_solve_continue`;
    the line reports pair-evals/s and ms per coverage solve (100 outer
    iterations).  The roofline of its all-pairs pass (8 FP32 operations and
    one exponential per pair: 2 subtractions and 2 FMA for the distance, 4
    FMA to accumulate) is reported for context; a field of 65536 pairs is a
    few microseconds, far from steady state."""
    import torch
    import torch.distributed as dist

    import oracle as orc
    from paper_2511_11514_b300 import binding as cov

    inst = wl.make_instance(w, seed=w.seed + rank)
    ctx = cov.Context(local_rank)
    dev = torch.device("cuda", local_rank)
    gmm = tuple(wl.f32_pair(v)[1] for v in inst.gmm)
    prob = cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, gmm=gmm, h=w.h)
    u = torch.as_tensor(inst.u0, dtype=torch.float64, device=dev).contiguous()
    s = cov.cov_solve(ctx, prob, 0, u)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        cov.cov_solve_continue(ctx, prob, 1, u, s)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.2)
    torch.cuda.profiler.start()
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        cov.cov_solve_continue(ctx, prob, 1, u, s)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)), world, dev)
    st, flags = ctx.device_status()
    if st != cov.COV_OK:
        raise SystemExit(f"device status {cov.status_string(st)} flags {flags}")
    pairs_step = w.T * w.T
    ms_per_step = total_ms / args.steps
    # the field alone: 20 calls captured in a CUDA graph, so that the device
    # time of a ~2 us field is measured rather than the host's call overhead
    x = s[1:, :2].float().contiguous()
    a_buf = torch.empty_like(x)
    cov.cov_field_svgd(ctx, x, w.h, gmm=gmm, out=a_buf)
    torch.cuda.synchronize()
    fg = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(fg, stream=side):
            for _ in range(20):
                cov.cov_field_svgd(ctx, x, w.h, gmm=gmm, out=a_buf)
    stream.wait_stream(side)
    fg.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fg.replay()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) / 20)
    field_ms = statistics.median(ts)
    del fg
    probe = cov.cov_probe_peaks(ctx, 4096)
    clk_hz = SM_MAX_MHZ_NOMINAL * 1e6
    fp32 = SM_COUNT_NOMINAL * FP32_LANES_PER_SM_CLK * clk_hz / 8
    mufu = SM_COUNT_NOMINAL * 32 * clk_hz
    peak = min(fp32, mufu)
    # end to end: controls and reference parameters from pinned host memory
    u_h = torch.as_tensor(inst.u0, dtype=torch.float64).pin_memory()
    u_out = torch.empty_like(u_h).pin_memory()
    s_out = torch.empty((w.T + 1, s.shape[1]), dtype=torch.float64).pin_memory()
    e_ms = []
    for k in range(args.e2e_steps + 2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        u.copy_(u_h, non_blocking=True)
        cov.cov_solve(ctx, prob, 1, u, s)
        u_out.copy_(u, non_blocking=True)
        s_out.copy_(s, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if k >= 2:
            e_ms.append(a.elapsed_time(b))
    e2e_ms = statistics.mean(e_ms)
    launches = count_library_launches(lambda: cov.cov_solve_continue(ctx, prob, 1, u, s))
    # one whole coverage solve from the initial controls on a context of its
    # own (workspace reserved before the clock starts): initial rollout,
    # gains, graph capture and every outer iteration; then the same solve
    # again on that context (graph and gains already there)
    solve = None
    if rank == 0:
        c2 = cov.Context(local_rank)
        n, m = wl.MODEL_DIMS[w.model]
        c2.reserve_for(w.T, 0, 2, n, m)
        u2 = torch.as_tensor(inst.u0, dtype=torch.float64, device=dev).contiguous()
        s2 = torch.empty_like(s)
        runs = []
        for _ in range(2):
            u2.copy_(torch.as_tensor(inst.u0, dtype=torch.float64))
            torch.cuda.synchronize()
            sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sa.record(stream)
            cov.cov_solve(c2, prob, w.n_outer, u2, s2)
            sb.record(stream)
            torch.cuda.synchronize()
            runs.append(sa.elapsed_time(sb))
        st2, fl2 = c2.device_status()
        c2.close()
        if st2 != cov.COV_OK:
            raise SystemExit(f"device status {cov.status_string(st2)} flags {fl2}")
        solve = {"outer_iterations": w.n_outer, "ms": runs[0], "ms_repeat": runs[1],
                 "how": "cov_solve from the initial controls on a fresh context (workspace reserved beforehand): "
                        "initial rollout, gains, graph capture, every outer iteration; ms_repeat: the same solve "
                        "again on that context; CUDA events on the stream"}
    if rank == 0:
        line = {"metric": METRIC, "value": job_value(world, pairs_step, args.steps, total_ms), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded Philox Gaussian-mixture reference)",
                "config": {"workload": w.name, "T": w.T, "d": 2, "h": w.h, "model": "single_integrator",
                           "reference": f"{w.gmm_K}-component Gaussian mixture (score in closed form)",
                           "pairs_per_step": pairs_step, "outer_iterations_per_solve": w.n_outer,
                           "ms_per_coverage_solve": solve["ms"] if solve else None,
                           "coverage_solve": solve,
                           "precision": "f32 field, f64 LQR and rollout",
                           "parallelism": f"{world} independent problems (one per GPU)" if world > 1 else "single GPU",
                           "l2": "flushed between steps (256 MiB write outside the per-step CUDA events)"},
                "roofline": {"bound": "alu", "achieved": pairs_step / (field_ms * 1e-3) / 1e9, "peak": peak / 1e9,
                             "unit": "Gpair/s", "frac": pairs_step / (field_ms * 1e-3) / peak, "traffic": None,
                             "kernel": "svgd_small_kernel (the one-launch Stein field, T <= 1024; cov_field_svgd, 20 calls in a CUDA graph)",
                             "peak_basis": "148 SMs x 2032 MHz x min(32 ex2, 128 FP32 lanes / 8 ops per pair)",
                             "note": f"one field = {pairs_step} pairs in {field_ms * 1e3:.1f} us: launch- and "
                                     "latency-bound, not graded against the roofline", "probe": probe},
                "clocks": clk,
                "e2e": {"value": pairs_step / (e2e_ms * 1e-3), "unit": UNIT,
                        "h2d_bytes_per_step": u_h.numel() * 8,
                        "d2h_bytes_per_step": u_out.numel() * 8 + s_out.numel() * 8, "ms_per_step": e2e_ms},
                "gpu_launches": launches * args.steps}
        if world == 1 and not args.no_cpu_baseline:
            orc.build()
            orc.set_threads(os.cpu_count() or 1)
            orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, 2, gmm=gmm, h=w.h)
            t0 = time.perf_counter()
            orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, w.n_outer, gmm=gmm, h=w.h)
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": w.n_outer * pairs_step / dt, "unit": UNIT, "cores": orc.get_threads(),
                                    "kind": "oracle", **host_cpu(),
                                    "sample": f"FP64 oracle: the whole coverage solve ({w.n_outer} outer "
                                              f"iterations) in {dt:.2f} s, {orc.get_threads()} threads",
                                    "ms_per_coverage_solve": dt * 1e3}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Batched form: independent double-integrator problems, T ~ U{128..4096},
    M ~ U{512..16384}, half Stein / half Sinkhorn (50 iterations), advanced by
    one CUDA-graph launch per outer iteration, against the same problems solved
    one by one with cov_solve on the same GPU.  Under N ranks every rank takes
    the problems `assign_problems` gives it (by pair count) and advances them
    as its own batch; the job is timed by the slowest rank (weak scaling: the
    batch grows with N, `args.batched` problems per rank)."""
    import torch
    import torch.distributed as dist

    from paper_2511_11514_b300 import binding as cov

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    all_insts = wl.make_batch(args.batched * world, seed=0)
    mine = assign_problems([i.wl.pairs_per_field for i in all_insts], world)[rank]
    insts = [all_insts[k] for k in mine]
    ctx = cov.Context(local_rank)
    if args.batch_share:
        ctx.set_option(cov.OPT_BATCH_SHARE, args.batch_share)
    dev = torch.device("cuda", local_rank)
    ys = [torch.as_tensor(i.y, dtype=torch.float32, device=dev) if i.y is not None else None for i in insts]
    probs = []
    for i, y in zip(insts, ys):
        w = i.wl
        if w.field == wl.FIELD_SVGD:
            probs.append(cov.make_problem(w.model, w.T, w.dt, i.s0, w.field, i.Q, i.R, w.eta, gmm=i.gmm, h=w.h))
        else:
            probs.append(cov.make_problem(w.model, w.T, w.dt, i.s0, w.field, i.Q, i.R, w.eta, y=y, eps=w.eps,
                                          n_iter=w.n_iter))
    pairs = sum(i.wl.pairs_per_field for i in insts)
    pairs_job = sum(i.wl.pairs_per_field for i in all_insts)
    us = [torch.as_tensor(i.u0, dtype=torch.float64, device=dev) for i in insts]
    t0 = time.perf_counter()
    ss = cov.cov_solve_batched(ctx, probs, max(1, args.warmup), us)  # includes graph capture
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    clocks = Clocks(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    cov.cov_solve_batched(ctx, probs, args.steps, us, ss)
    b.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    batched_ms = max_over_ranks(a.elapsed_time(b), world, dev)
    clk = clocks.stop()
    st, flags = ctx.device_status()
    if st != cov.COV_OK:
        raise SystemExit(f"device status {cov.status_string(st)} flags {flags}")
    # one by one: cov_solve per problem (its graph captured in an untimed call)
    one_ms = 0.0
    for pr, i in zip(probs, insts):
        u1 = torch.as_tensor(i.u0, dtype=torch.float64, device=dev)
        cov.cov_solve(ctx, pr, 1, u1)
        a.record()
        cov.cov_solve(ctx, pr, args.steps, u1)
        b.record()
        torch.cuda.synchronize()
        one_ms += a.elapsed_time(b)
    one_ms = max_over_ranks(one_ms, world, dev)
    value = pairs_job * args.steps / (batched_ms * 1e-3)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": batched_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded Philox mixtures, uneven sizes)",
                "config": {"workload": f"batched_double_integrator_{args.batched}_problems_per_gpu",
                           "problems": args.batched * world, "problems_rank0": len(insts),
                           "T": "U{128..4096}", "M": "U{512..16384}",
                           "fields": "half Stein (h = 0.05), half Sinkhorn (eps = 0.005, 50 iterations)",
                           "pairs_per_step": pairs_job, "pairs_per_step_rank0": pairs,
                           "graph_capture_and_setup_s": setup_s,
                           "parallelism": (f"{world} ranks, problems assigned by pair count (longest first), no "
                                           "data-path collective" if world > 1 else "single GPU"),
                           "l2": "not flushed (the batch working set, ~GBs, exceeds L2)"},
                "one_by_one": {"value": pairs_job * args.steps / (one_ms * 1e-3), "unit": UNIT,
                               "ms_per_step": one_ms / args.steps,
                               "how": "cov_solve on each problem in turn, same GPU, same context, graphs "
                                      "pre-captured"},
                "batched_speedup": one_ms / batched_ms, "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_adjoint(args):
    """Differentiation workload: the coverage loss (Sinkhorn divergence of the
    final positions to a held-out 4-component mixture) after K = 20 outer
    iterations (T = 2048, M = 8192, eps = 0.005, 50 iterations), differentiated
    with respect to the reference mixture's means, log-sigmas and logits
    (samples by reparameterisation) and the initial state.  A step is one
    forward (reparameterisation, checkpointed solve, loss) and one backward
    (loss gradient, reverse sweep, reparameterisation chain), each timed with
    CUDA events; the line reports the backward / forward time ratio."""
    import torch

    from paper_2511_11514_b300 import autograd as ag
    from paper_2511_11514_b300 import binding as cov

    torch.cuda.set_device(0)
    w = wl.ADJOINT_DOUBLE_T2048
    if args.adjoint_outer:
        w = dataclasses.replace(w, n_outer=args.adjoint_outer)
    inst = wl.make_instance(w)
    ctx = cov.Context(0)
    # the loss runs on its own context: a field call on the solve's context
    # would overwrite the Riccati gains cov_solve caches in its workspace
    lctx = cov.Context(0)
    dev = torch.device("cuda", 0)
    gw, gmu, gsig = inst.gmm
    mu = torch.tensor(gmu, dtype=torch.float32, device=dev, requires_grad=True)
    log_sigma = torch.tensor(np.log(gsig), dtype=torch.float32, device=dev, requires_grad=True)
    logits = torch.tensor(np.log(gw), dtype=torch.float32, device=dev, requires_grad=True)
    s0 = torch.tensor(inst.s0, dtype=torch.float64, requires_grad=True)
    u0 = torch.as_tensor(inst.u0, dtype=torch.float64, device=dev)
    xi = ag.standard_draws(w.M, 2, seed=w.seed + 2000, device=dev)
    lw, lmu, lsig = wl.gmm_params(4, w.extra["loss_seed"])
    y_loss = torch.as_tensor(wl.f32_pair(wl.gmm_samples(lw, lmu, lsig, w.extra["loss_M"], w.extra["loss_seed"] + 1000))[1],
                             dtype=torch.float32, device=dev)
    eps_l, it_l = w.extra["loss_eps"], w.extra["loss_iters"]
    q_ref = ag.reference_self_potential(lctx, y_loss, eps_l, it_l)
    spec = dict(model=w.model, dt=w.dt, Q=inst.Q, R=inst.R, eta=w.eta, eps=w.eps, n_iter=w.n_iter,
                n_outer=w.n_outer)

    def forward():
        y, b = ag.gmm_reference(mu, log_sigma, logits, xi)
        s_K = ag.CoverageSolve.apply(y, b, s0, u0, spec, ctx)
        return ag.SinkhornLoss.apply(s_K[1:, :2].float().contiguous(), y_loss, eps_l, it_l, lctx, q_ref)

    params = (mu, log_sigma, logits, s0)
    for _ in range(max(1, args.warmup)):
        for p in params:
            p.grad = None
        forward().backward()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees the timed steps only
    fw, bw, losses = [], [], []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(args.steps):
        for p in params:
            p.grad = None
        torch.cuda.synchronize()
        ev[0].record()
        L = forward()
        ev[1].record()
        L.backward()
        ev[2].record()
        torch.cuda.synchronize()
        fw.append(ev[0].elapsed_time(ev[1]))
        bw.append(ev[1].elapsed_time(ev[2]))
        losses.append(float(L.detach()))
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    st, flags = ctx.device_status()
    if st != cov.COV_OK:
        raise SystemExit(f"device status {cov.status_string(st)} flags {flags}")
    f_ms, b_ms = statistics.median(fw), statistics.median(bw)
    pairs_fwd = w.n_outer * w.pairs_per_field

    # roofline of the reverse all-pairs kernel (adj_kernel, column sums): per
    # Sinkhorn iteration the reverse sweep evaluates 2TM + T^2 pairs.  Its time
    # per iteration is that of the backward of one recorded outer iteration
    # (no forward Sinkhorn inside: the records are replayed) as
    # (t(n_hi) - t(n_lo)) / (n_hi - n_lo) in the Sinkhorn iteration count.
    def reverse_per_iter_ms(T, M, lo, hi, reps):
        inst_r = wl.make_instance(wl.SINKHORN_DOUBLE_T4096, T=T, M=M)
        wr = inst_r.wl
        yr = torch.as_tensor(inst_r.y, dtype=torch.float32, device=dev)
        u0r = torch.as_tensor(inst_r.u0, dtype=torch.float64, device=dev)
        sbar = torch.as_tensor(wl.rng(w.seed + 3001).standard_normal((T + 1, 4)), dtype=torch.float64, device=dev)
        rctx = cov.Context(0)
        ts = {}
        for n in (lo, hi):
            P = cov.make_problem(wr.model, T, wr.dt, inst_r.s0, wr.field, inst_r.Q, inst_r.R, wr.eta, y=yr,
                                 eps=w.eps, n_iter=n)
            _, hist, token, P2 = cov.grad_forward(rctx, P, 1, u0r, yr)
            cov.grad_backward(rctx, P2, 1, u0r, sbar, hist, token, yr)   # warm (graph capture)
            samples = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                cov.grad_backward(rctx, P2, 1, u0r, sbar, hist, token, yr)
                e1.record()
                torch.cuda.synchronize()
                samples.append(e0.elapsed_time(e1))
            ts[n] = statistics.median(samples)
        st_r, fl_r = rctx.device_status()
        if st_r != cov.COV_OK:
            raise SystemExit(f"device status {cov.status_string(st_r)} flags {fl_r}")
        rctx.close()
        return (ts[hi] - ts[lo]) / (hi - lo)

    rev_ms = max(reverse_per_iter_ms(w.T, w.M, 10, 50, 5), 1e-9)
    rev_pairs = 2 * w.T * w.M + w.T * w.T
    adj_peak = SM_COUNT_NOMINAL * SM_MAX_MHZ_NOMINAL * 1e6 * FP32_LANES_PER_SM_CLK / 6
    achieved = rev_pairs / (rev_ms * 1e-3)
    # the same at a size where a launch is long enough to reach steady state
    TL, ML = 16384, 65536
    rev_l = max(reverse_per_iter_ms(TL, ML, 2, 6, 3), 1e-9)
    achieved_l = (2 * TL * ML + TL * TL) / (rev_l * 1e-3)
    line = {"metric": "backward/forward time ratio of the coverage-loss gradient", "value": b_ms / f_ms,
            "unit": "x", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": f_ms + b_ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 fields, f64 LQR/rollout", "data": "synthetic (seeded Philox mixtures)",
            "config": {"workload": w.name, "T": w.T, "M": w.M, "eps": w.eps, "n_iter": w.n_iter,
                       "n_outer": w.n_outer, "loss": f"S_eps to held-out 4-GMM, M={w.extra['loss_M']}, "
                       f"eps={eps_l}, {it_l} iterations", "params": "means, log-sigmas, logits, s0",
                       "pairs_forward": pairs_fwd, "l2": "not flushed (forward and backward alternate)"},
            "ms_forward": f_ms, "ms_backward": b_ms,
            "roofline": {"bound": "alu", "kernel": "adj_kernel (reverse column sums)", "achieved": achieved,
                         "peak": adj_peak, "unit": "pair-evals/s", "frac": achieved / adj_peak, "traffic": None,
                         "peak_basis": "148 SMs x 2032 MHz x 128 FP32 lanes / 6 FP32 ops per pair (add of the "
                                       "row term, 2 FMA exponent, 3 FMA accumulation; derived from unit counts and "
                                       "clocks; ex2 at 32/clk/SM is not binding)",
                         "how": "backward of one recorded outer iteration, (t(50) - t(10)) / 40 Sinkhorn "
                                "iterations; 2TM + T^2 pairs per reverse iteration"},
            "ms_per_reverse_sinkhorn_iteration": rev_ms,
            "roofline_large": {"bound": "alu", "T": TL, "M": ML, "achieved": achieved_l, "peak": adj_peak,
                               "unit": "pair-evals/s", "frac": achieved_l / adj_peak,
                               "ms_per_reverse_sinkhorn_iteration": rev_l, "how": "(t(6) - t(2)) / 4"},
            "forward_pairs_per_s": pairs_fwd / (f_ms * 1e-3), "loss": losses[-1],
            "grad_norms": {"mu": float(mu.grad.norm()), "log_sigma": float(log_sigma.grad.norm()),
                           "logits": float(logits.grad.norm()), "s0": float(s0.grad.norm())},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    lctx.close()
    ctx.close()
    return 0


def run_variants(args):
    """Equal-accuracy comparison of the Sinkhorn variants at eps = 0.002 on the
    benchmark's sizes (T = 4096 samples of the initial double-integrator
    trajectory, M = 16384 mixture samples): the field after n iterations is
    compared with the converged field (4000 cold iterations), for the paper's
    cold iteration, eps-scaling (eps_t = max(eps, 0.08 * 0.85^t)) and a warm
    start from the converged potentials of the trajectory one outer
    iteration earlier.  Reports, per variant, the iterations needed to reach
    a relative field error of 1e-2 and 1e-3 and the time per iteration."""
    import torch

    from paper_2511_11514_b300 import binding as cov

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = wl.SINKHORN_DOUBLE_T4096
    inst = wl.make_instance(w)
    ctx = cov.Context(0)
    eps, e0, dec = 0.002, 0.08, 0.85
    y = torch.as_tensor(inst.y, dtype=torch.float32, device=dev)
    P = cov.make_problem(w.model, w.T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, y=y, eps=eps, n_iter=50)
    u = torch.as_tensor(inst.u0, dtype=torch.float64, device=dev)
    s_prev = cov.cov_solve(ctx, P, 4, u).clone()                  # a trajectory a few iterations in
    s_cur = cov.cov_solve_continue(ctx, P, 1, u, s_prev.clone())  # and the one after it
    x_prev = s_prev[1:, :2].float().contiguous()
    x = s_cur[1:, :2].float().contiguous()
    a_ref, _, _, _ = cov.cov_field_sinkhorn(ctx, x, y, eps, 4000)
    _, f_w, g_w, p_w = cov.cov_field_sinkhorn(ctx, x_prev, y, eps, 4000)
    ref_norm = float(a_ref.double().norm())

    def err(a):
        return float((a.double() - a_ref.double()).norm()) / ref_norm

    grid = [5, 10, 15, 20, 25, 30, 40, 50, 60, 80, 100, 130, 160, 200, 260, 330, 420, 540, 700, 900, 1200]
    curves = {"cold": [], "eps_scaling": [], "warm": []}
    for n in grid:
        curves["cold"].append(err(cov.cov_field_sinkhorn(ctx, x, y, eps, n)[0]))
        curves["eps_scaling"].append(err(cov.cov_field_sinkhorn_annealed(ctx, x, y, eps, n, e0, dec)[0]))
        curves["warm"].append(err(cov.cov_field_sinkhorn(ctx, x, y, eps, n, f=f_w.clone(), g=g_w.clone(),
                                                          p=p_w.clone(), warm=True)[0]))

    def first_below(c, tol):
        for n, e in zip(grid, c):
            if e <= tol:
                return n
        return None

    stream = torch.cuda.current_stream()

    def per_iter_ms(fn):
        ts = []
        for n in (20, 120):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            fn(n)
            a.record(stream)
            fn(n)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return (ts[1] - ts[0]) / 100

    t_cold = per_iter_ms(lambda n: cov.cov_field_sinkhorn(ctx, x, y, eps, n, field=False))
    t_scaled = per_iter_ms(lambda n: cov.cov_field_sinkhorn_annealed(ctx, x, y, eps, n, e0, dec, field=False))
    st, flags = ctx.device_status()
    if st != cov.COV_OK:
        raise SystemExit(f"device status {cov.status_string(st)} flags {flags}")
    res = {v: {"iters_to_1e-2": first_below(c, 1e-2), "iters_to_1e-3": first_below(c, 1e-3)}
           for v, c in curves.items()}
    n_c, n_s, n_w = (res[v]["iters_to_1e-3"] for v in ("cold", "eps_scaling", "warm"))
    line = {"metric": "Sinkhorn iterations to a 1e-3 field error at eps = 0.002 (cold / eps-scaled / warm)",
            "value": {"cold": n_c, "eps_scaling": n_s, "warm": n_w}, "unit": "iterations",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic (seeded Philox mixture)",
            "config": {"workload": f"{w.name} trajectory, eps = 0.002", "T": w.T, "M": w.M,
                       "eps_schedule": f"max(eps, {e0} * {dec}^t)",
                       "warm": "converged potentials of the previous outer iteration's trajectory",
                       "reference": "4000 cold iterations"},
            "variants": res, "grid": grid, "relative_field_error": curves,
            "ms_per_iteration": {"cold": t_cold, "eps_scaling": t_scaled}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_horizon_sweep(args):
    """Coverage-solve time against the horizon T, GPU (this library, one
    B300) against the FP64 oracle on the host cores, in the shape of the
    paper's timing study (solve time vs horizon, GPU vs CPU).  The paper's
    differential-drive and aircraft models are not specified; the Stein
    points use the unicycle (the differential drive's kinematic form) with a
    3-component mixture, h = 0.05, eta = 1e-3, K = 100 outer iterations; the
    Sinkhorn points the double integrator with M = T reference samples of an
    8-component mixture, eps = 0.005, 50 iterations, eta = 0.5, K = 20 outer
    iterations.  GPU: `cov_solve` for K outer iterations (CUDA events, after
    an untimed call that captures the graph and caches the gains).  Oracle
    (the CPU baseline of this sweep): timed over k <= K outer iterations,
    k chosen so that each point costs ~1 s of host time, and scaled to K
    ("extrapolated" where k < K)."""
    import torch

    import oracle as orc
    from paper_2511_11514_b300 import binding as cov

    orc.build()
    orc.set_threads(os.cpu_count() or 1)
    torch.cuda.set_device(0)
    ctx = cov.Context(0)
    dev = torch.device("cuda", 0)
    points = []
    specs = [("svgd", T) for T in (100, 256, 500, 1000, 2000, 5000, 10000)] + \
            [("sinkhorn", T) for T in (100, 200, 500, 1000, 2500)]
    for kind, T in specs:
        if kind == "svgd":
            w = dataclasses.replace(wl.SVGD_SINGLE_T256, name=f"svgd_unicycle_T{T}", model=wl.UNICYCLE, T=T,
                                    dt=0.01, n_outer=100)
            inst = wl.make_instance(w)
            gmm = tuple(wl.f32_pair(v)[1] for v in inst.gmm)
            prob = cov.make_problem(w.model, T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, gmm=gmm, h=w.h)
            oracle_kw = dict(gmm=gmm, h=w.h)
            pairs_outer = T * T
        else:
            w = dataclasses.replace(wl.SINKHORN_DOUBLE_T4096, name=f"sinkhorn_double_integrator_T{T}", T=T, M=T,
                                    n_outer=20)
            inst = wl.make_instance(w)
            y = torch.as_tensor(inst.y, dtype=torch.float32, device=dev)
            prob = cov.make_problem(w.model, T, w.dt, inst.s0, w.field, inst.Q, inst.R, w.eta, y=y, eps=w.eps,
                                    n_iter=w.n_iter)
            oracle_kw = dict(y=inst.y, eps=w.eps, n_iter=w.n_iter)
            pairs_outer = w.n_iter * (2 * T * T + T * T) + (T * T + T * T)
        K = w.n_outer
        u0 = torch.as_tensor(inst.u0, dtype=torch.float64, device=dev)
        u = u0.clone()
        cov.cov_solve(ctx, prob, K, u)        # graph capture, gains
        ts = []
        for _ in range(3):
            u.copy_(u0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            cov.cov_solve(ctx, prob, K, u)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        gpu_ms = statistics.median(ts)
        # oracle: one outer iteration to size the sample, then k of them
        t0 = time.perf_counter()
        orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, 1, **oracle_kw)
        one = time.perf_counter() - t0
        k = int(max(1, min(K, round(1.0 / max(one, 1e-6)))))
        t0 = time.perf_counter()
        orc.solve(w.model, w.dt, inst.s0, inst.u0, w.field, inst.Q, inst.R, w.eta, k, **oracle_kw)
        cpu_ms = (time.perf_counter() - t0) * 1e3 * K / k
        points.append({"field": kind, "T": T, "M": T if kind == "sinkhorn" else 0, "outer_iterations": K,
                       "gpu_ms_per_solve": gpu_ms, "cpu_ms_per_solve": cpu_ms,
                       "cpu_outer_iterations_timed": k, "cpu_extrapolated": k < K,
                       "speedup": cpu_ms / gpu_ms, "gpu_pair_evals_per_s": K * pairs_outer / (gpu_ms * 1e-3)})
        print(json.dumps(points[-1]), file=sys.stderr, flush=True)
    st, flags = ctx.device_status()
    if st != cov.COV_OK:
        raise SystemExit(f"device status {cov.status_string(st)} flags {flags}")
    ctx.close()
    line = {"metric": "coverage solve time vs horizon, GPU vs FP64 oracle (context)", "value": None, "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32 fields, f64 LQR/rollout",
            "data": "synthetic (seeded Philox mixtures)", "cpu_cores": orc.get_threads(), **host_cpu(), "points": points}
    print(json.dumps(line), flush=True)
    return 0


def run_lqr_sweep(args):
    """The LQR step alone against the horizon: `cov_lqr_track` (the
    parallel-in-time Riccati recursion and the two affine scans, FP64) on the
    linearisation of a unicycle trajectory (speeds and turn rates varying
    along the horizon, dt = 0.01, position-only Q, R = 0.01 I), CUDA events
    over `--steps` calls after `--warmup` untimed ones."""
    import torch

    from paper_2511_11514_b300 import binding as cov

    torch.cuda.set_device(0)
    ctx = cov.Context(0)
    dev = torch.device("cuda", 0)
    points = []
    for T in (int(t) for t in args.lqr_sweep.split(",") if t.strip()):
        dt = 0.01
        s0, u = wl.unicycle_init(T, dt)
        ts = np.arange(T)
        u = u + np.stack([0.05 * np.sin(ts / 500.0), 0.5 * np.cos(ts / 800.0)], 1)
        ud = torch.as_tensor(u, dtype=torch.float64, device=dev)
        s = cov.cov_rollout(ctx, wl.UNICYCLE, s0, ud, dt)
        A, B = cov.cov_linearize(ctx, wl.UNICYCLE, s, ud, dt)
        abar = torch.zeros((T, 3), dtype=torch.float64, device=dev)
        abar[:, :2] = 0.05
        Q, R = wl.coverage_Q(wl.UNICYCLE), 0.01 * np.eye(2)
        for _ in range(max(1, args.warmup)):
            cov.cov_lqr_track(ctx, A, B, Q, R, abar)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            cov.cov_lqr_track(ctx, A, B, Q, R, abar)
        b.record()
        torch.cuda.synchronize()
        points.append({"T": T, "us_per_lqr_step": a.elapsed_time(b) / args.steps * 1e3})
    st, flags = ctx.device_status()
    if st != cov.COV_OK:
        raise SystemExit(f"device status {cov.status_string(st)} flags {flags}")
    print(json.dumps({"metric": "LQR step time vs horizon (context)", "value": None, "unit": "us",
                      "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic unicycle trajectory",
                      "steps": args.steps, "warmup": args.warmup, "points": points}))


def main():
    args = parse_args()
    if args.lqr_sweep:
        return run_lqr_sweep(args)
    if args.horizon_sweep:
        return run_horizon_sweep(args)
    if args.variants:
        return run_variants(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.field_profile:
        return run_field_profile(args)
    if args.batched:
        return run_batched(args)
    if args.adjoint:
        return run_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
