"""The multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1) agree on the
slowest rank's step time and on the whole-job value (weak scaling: every rank runs its own
copy of the workload, no data-path collective)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    local_ms = [12.5, 20.0][rank]
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (ms, bench.job_value(world, 1000, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_and_value():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        ms, value = out[r]
        assert ms == 20.0
        assert value == pytest.approx(2 * 5 * 1000 / 20e-3)


def test_single_rank_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.job_value(1, 100, 2.0) == pytest.approx(5 * 100 / 2e-3)
