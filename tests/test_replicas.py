"""The multi-GPU path of bench.py is replicas only (a cloud is never
sharded): each rank samples its own scene and the job's value is every
rank's points over the slowest rank's time.  This checks that aggregation
over two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 2.0 if rank == 1 else 1.0  # rank 1 is the slow one
        t, v = bench.whole_job(local, points_per_rank=1_000_000, world=world, device="cpu")
        out[rank] = (t, v)
    finally:
        dist.destroy_process_group()


def test_whole_job_takes_max_time_and_all_points():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == pytest.approx(2.0)
        assert v == pytest.approx(2 * 1_000_000 / 2.0 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    t, v = bench.whole_job(0.5, 1_000_000, 1)
    assert t == 0.5 and v == pytest.approx(2.0)
