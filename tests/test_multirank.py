"""Host-side logic of the N > 1 benchmark path, with world size 2 on the gloo
backend (CPU): each rank runs its own replica of the step ("replicas only":
the SpMV path has no data-path exchange in this build), the reported time is
the maximum over ranks, and the value is the whole job's throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        elapsed = [12.5, 20.0][rank]            # the second rank is the slow one
        got = bench.max_over_ranks(elapsed, torch.device("cpu"))
        dist.barrier()
        out[rank] = (got, bench.whole_job_gbs(world, 1_000_000_000, got / 10))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    # 2 ranks x 1 GB per step at 2 ms per step = 1000 GB/s
    assert abs(res[0][1] - 1000.0) < 1e-9
