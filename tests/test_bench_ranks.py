"""The benchmark's multi-rank aggregation, run as two gloo ranks on the CPU:
each root slot takes the slowest rank's time and the ranks' summed edges."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_root = np.array([1.0, 2.0, 4.0]) * (rank + 1)       # rank 1 is slower
    m_c = np.array([100.0, 200.0, 400.0]) * (rank + 1)
    step_ms = np.array([10.0 * (rank + 1)])
    out = bench.aggregate_ranks(t_root, m_c, step_ms, world, torch.device("cpu"))
    q.put((rank, [x.tolist() if hasattr(x, "tolist") else x for x in out]))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    t_job, m_job, ms_step, value = res[0]
    assert t_job == [2.0, 4.0, 8.0]              # max over ranks
    assert m_job == [300.0, 600.0, 1200.0]       # sum over ranks
    assert ms_step == 20.0
    g = np.array(m_job) / (np.array(t_job) * 1e-3) / 1e9
    assert abs(value - len(g) / np.sum(1 / g)) < 1e-12
    assert res[1] == res[0]
