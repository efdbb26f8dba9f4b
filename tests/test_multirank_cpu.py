"""The N > 1 host logic of bench.py on CPU: two gloo ranks (127.0.0.1).

* the job time is the maximum over ranks (what every rank reports);
* the 64-box replica workload is split by LPT on atom counts: every box on
  exactly one rank, the same split on every rank, loads within the LPT
  bound (max load <= mean load + largest box).
"""
import os
import socket
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import bench                                  # noqa: E402
from paper_2212_08284_gb300 import synth      # noqa: E402


def test_lpt_partition_covers_and_balances():
    costs = [int(c) for c in synth.replica_sizes(64)]
    for nparts in (1, 2, 3, 4, 8):
        parts = bench.lpt_partition(costs, nparts)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / nparts + max(costs)
    # a hand-checked small case: 7, 5, 4, 3, 2 over 2 parts -> {7, 3, 2} {5, 4}... by LPT:
    # 7 -> p0 (7); 5 -> p1 (5); 4 -> p1 (9); 3 -> p0 (10); 2 -> p1 (11)
    assert bench.lpt_partition([7, 5, 4, 3, 2], 2) == [[0, 3], [1, 2, 4]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        parts = bench.lpt_partition([int(c) for c in synth.replica_sizes(64)], world)
        dist.barrier()
        q.put((rank, t, parts[rank], parts))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_split():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == res[1][1] == 2.5
    assert res[0][3] == res[1][3]
    assert sorted(res[0][2] + res[1][2]) == list(range(64))
