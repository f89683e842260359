"""bench.py --gpus N runs N independent replicas (seed = rank) and reduces
only the timing: the slowest rank's time and the sum of all ranks' updates.
That reduction runs here on the CPU with two gloo ranks."""

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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, upd = bench.combine_ranks(10.0 + rank, 1000.0 * (rank + 1), torch.device("cpu"), world)
    # every replica draws its own seeded problem
    import workloads as W
    rho = W.riemann_quadrants(nx=8, ny=8, nv=8, seed=rank)["fields"]["rho"]
    out[rank] = (ms, upd, float(rho.sum()))
    dist.destroy_process_group()


def test_two_gloo_replicas_reduce_time_and_updates():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert out[0][:2] == (11.0, 3000.0) and out[1][:2] == (11.0, 3000.0)
    assert out[0][2] != out[1][2]          # different seeds, different data


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(5.0, 7, torch.device("cpu"), 1) == (5.0, 7.0)
