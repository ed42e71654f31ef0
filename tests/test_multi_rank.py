"""Multi-rank timing of bench.py on CPU: two gloo ranks over 127.0.0.1.

The benchmark runs one independent replica per GPU; the whole-job value
divides every rank's frames by the slowest rank's time.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [40.0, 50.0][rank]          # rank 1 is the slower replica
    frames_local = [900 * 10, 900 * 10][rank]
    ms, value = bench.combine_ranks(torch, dist, ms_local, frames_local, world, torch.device("cpu"))
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_all_frames():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, value = res[rank]
        assert ms == 50.0
        assert abs(value - 2 * 900 * 10 / 0.050) < 1e-6


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.combine_ranks(torch, None, 25.0, 900, 1, torch.device("cpu"))
    assert ms == 25.0 and value == 900 / 0.025
