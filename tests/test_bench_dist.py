"""Multi-process host logic of bench.py on CPU (gloo, world size 2).

The benchmark runs one independent replica per rank (the solve itself has no
exchange step on one GPU per replica); what the ranks share is the barrier
before and after the timed region and the max-over-ranks of the elapsed time.
Both are exercised here with two gloo ranks, as is the rule that only rank 0
of the reference arm does work.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import torch.distributed as dist

    class A:
        gpus = ws
    got_ws, got_rank, _ = bench.dist_setup(A())
    bench.barrier(got_ws)
    m = bench.max_over_ranks(got_ws, 10.0 + 5.0 * got_rank)
    bench.barrier(got_ws)
    q.put((got_rank, got_ws, m))
    dist.destroy_process_group()


def test_two_ranks_barrier_and_max():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 15.0), (1, 2, 15.0)]


def test_reference_arm_runs_on_rank0_only(capsys):
    import bench

    class A:
        gpus, steps, warmup = 2, 1, 0
    bench.run_reference(A(), 2, 1)  # rank 1: returns without work or output
    assert capsys.readouterr().out == ""
