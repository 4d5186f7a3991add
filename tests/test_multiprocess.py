"""The N-GPU form of the benchmark on the CPU: two `gloo` ranks run the host
logic of `bench.py --gpus 2` (each rank its own problem, the job timed by its
slowest rank, the value aggregated over ranks) without a GPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2511_11514_b300 import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, ws = bench.dist_env()
        local_ms = 100.0 + 25.0 * rank                     # rank 1 is the slower one
        total = bench.max_over_ranks(local_ms, ws)
        w = wl.SINKHORN_DOUBLE_T4096
        inst = wl.make_instance(w, T=64, M=64, seed=w.seed + r)  # each rank its own problem
        out.put((r, ws, total, bench.job_value(ws, w.pairs_per_field, 10, total), float(inst.y[0, 0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, t0, v0, y0), (r1, w1, t1, v1, y1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert t0 == t1 == 125.0                               # max over ranks
    from paper_2511_11514_b300 import workloads as wl
    pairs = wl.SINKHORN_DOUBLE_T4096.pairs_per_field
    assert v0 == pytest.approx(2 * pairs * 10 / 0.125)     # whole job: both ranks' pairs over the slowest time
    assert y0 != y1                                        # the ranks solve different problems
