"""The N > 1 benchmark path on the host: two gloo ranks on the CPU agree on the slowest rank's step
time and on the whole-job throughput (replicas process the same units, so the job's bytes scale
with the world size and its time is the max over ranks)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(1.5 + rank, world, torch.device("cpu"))  # rank 1 is the slow one
    q.put((rank, ms, bench.whole_job_gbs(3e9, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_aggregate():
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [2.5, 2.5]
    assert got[0][2] == pytest.approx(2 * 3e9 / 2.5e-3 / 1e9)  # 2400 GB/s over both replicas


def test_world_one_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.25, 1, None) == 1.25
    assert bench.whole_job_gbs(1e9, 1, 1.0) == pytest.approx(1000.0)
