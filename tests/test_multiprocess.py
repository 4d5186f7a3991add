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


def _batch_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from paper_2511_11514_b300 import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, _, ws = bench.dist_env()
        insts = wl.make_batch(20 * ws, seed=0, T_range=(32, 256), M_range=(32, 256))
        costs = [i.wl.pairs_per_field for i in insts]
        mine = bench.assign_problems(costs, ws)[r]
        # every rank computes the same partition; gather it to check
        got = [None] * ws
        dist.all_gather_object(got, mine)
        load = float(sum(costs[k] for k in mine))
        t = torch.tensor([load], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        out.put((r, got, load, float(t.item()), costs))
    finally:
        dist.destroy_process_group()


def test_batched_problems_partition_over_two_gloo_ranks():
    """`bench.py --batched` under two ranks: each rank takes the problems the
    deterministic assignment gives it (no collective needed to agree on the
    partition); together they cover the batch exactly once and the heavier
    rank carries at most the lighter one's work plus one problem."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, g0, l0, m0, costs), (_, g1, l1, m1, _) = res
    assert g0 == g1                                   # both ranks computed the same partition
    idx = sorted(g0[0] + g0[1])
    assert idx == list(range(len(costs)))             # every problem exactly once
    assert m0 == m1 == max(l0, l1)
    assert abs(l0 - l1) <= max(costs)


def test_assignment_balances_by_cost():
    sys.path.insert(0, ROOT)
    import bench
    parts = bench.assign_problems([5, 1, 1, 1, 1, 1], 2)
    assert parts == [[0], [1, 2, 3, 4, 5]]
    # longest first, each to the least-loaded rank: loads 3 | 3 | 2, then 3 | 3 | 4, then 5 | 3 | 4
    assert bench.assign_problems([3, 3, 2, 2, 2], 3) == [[0, 4], [1], [2, 3]]
