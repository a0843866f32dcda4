"""Host logic of the multi-GPU replicas path of bench.py, on CPU with two gloo ranks:
every rank ends with the slowest rank's time, the whole-job rate counts every replica's
bytes over that time, and the reference arm does its work on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1.5, 2.5][rank]
    ms = bench.max_over_ranks(dist, local_ms, torch.device("cpu"))
    value = bench.whole_job_gbs(world, 4.0e9, ms * 1e-3)
    out[rank] = (ms, value)

    class Args:
        steps, warmup, gpus = 1, 0, world
    if rank != 0:
        # the reference arm returns at once on ranks other than 0 (no work, no output)
        assert bench.run_reference(Args(), rank, world) is None
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    # two replicas of 4 GB each in 2.5 ms
    assert res[0][1] == pytest.approx(2 * 4.0e9 / 2.5e-3 / 1e9)


def test_single_process_is_unchanged():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.25, None) == 3.25
    assert bench.whole_job_gbs(1, 1e9, 1e-3) == pytest.approx(1000.0)
