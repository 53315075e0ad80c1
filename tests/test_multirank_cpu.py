"""The bench's multi-rank host logic on CPU: two gloo ranks (127.0.0.1), each timing
its own replica; the whole-job value is all ranks' columns over the slowest rank's
time, every rank sees the same maximum, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    dist = bench.Dist()
    dist.init("gloo")
    ms_local = 10.0 * (rank + 1)           # rank 1 is the slowest
    value, ms = bench.aggregate(dist, 256, ms_local)
    dist.barrier()

    class Args:
        steps, warmup, cpu_seconds, gpus = 1, 0, 1.0, world
    ran = bench.run_reference(Args(), dist) if rank != 0 else "skipped"
    out[rank] = (value, ms, ran)
    dist.close()


def test_two_gloo_ranks_aggregate_and_reference_on_rank0_only():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, ms, ran = res[rank]
        assert ms == 20.0                       # the slowest rank's time, seen by every rank
        assert value == pytest.approx(world * 256 / 0.020)
    assert res[1][2] is None                    # the reference arm does no work off rank 0
