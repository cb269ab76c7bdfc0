"""The multi-rank path of bench.py on CPU: two gloo ranks, each timing its own
replica, reduce the step time by max and report the whole-job rate."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + rank                    # rank 1 is the slower replica
    ms_max = bench.reduce_max(ms, dist, "cpu")
    q.put((rank, ms_max, bench.whole_job_rate(1000, world, ms_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_by_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, rate in res:
        assert ms_max == 11.0
        assert rate == pytest.approx(2 * 1000 / 0.011)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(100, 1, 1.0) == pytest.approx(1e5)
