"""Multi-rank host logic of bench.py, on CPU with the gloo backend (world size 2).

bench.py runs one process per GPU under torchrun.  Its data path has no
collective: the headline solve runs as independent replicas and the
512-problem batch is sharded by a longest-processing-time partition.  The
only cross-rank steps are host-side: the slowest rank's time (max over
ranks), the units all ranks processed (sum over ranks), and the reference
arm running on rank 0 alone.  These are exercised here without a GPU.
"""
import argparse
import io
import json
import os
import socket
from contextlib import redirect_stdout

import pytest

import bench
import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank)  # the slower rank is rank 1
        u = bench.sum_over_ranks(10.0 * (rank + 1))
        probs = workloads.batch_problems(512)
        costs = [bench.problem_cost(bp) for bp in probs]
        mine = bench.lpt_partition(costs, world)[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, t, u, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, t, u, gathered in out:
        assert t == 2.5           # max over ranks
        assert u == 30.0          # sum over ranks
        assert gathered == out[0][3]
    parts = out[0][3]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(512))  # disjoint and complete


def test_lpt_partition_balance():
    probs = workloads.batch_problems(512)
    costs = [bench.problem_cost(bp) for bp in probs]
    for k in (1, 2, 3, 4, 8):
        parts = bench.lpt_partition(costs, k)
        assert sorted(i for p in parts for i in p) == list(range(512))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy LPT: every load is within one largest item of the mean
        assert max(loads) - sum(loads) / k <= max(costs) + 1e-9


def test_single_process_reductions_are_identity():
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.sum_over_ranks(7.0) == 7.0


def _ref_args(**kw):
    a = dict(gpus=1, steps=1, warmup=1, impl="reference", ref_n=8, cpu_n=8, no_cpu=True, no_fp64=True,
             no_e2e=True, unfused=False, n=256, workload="c3")
    a.update(kw)
    return argparse.Namespace(**a)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import oracle
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    def boom(*a, **k):
        raise AssertionError("a non-zero rank must not run the oracle")

    monkeypatch.setattr(oracle, "solve_unbounded", boom)
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(_ref_args()) == 0
    assert buf.getvalue() == ""


def test_reference_arm_line(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(_ref_args()) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["config"] == bench.c3_config(bench.N, 1)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
