"""The multi-GPU benchmark path runs independent replicas; its only
cross-rank step is the max-over-ranks reduction of the timed region. That
aggregation is exercised here with world_size 2 on the gloo backend (CPU)."""

import importlib.util
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ms_local = [100.0, 125.0][rank]  # rank 1 is the slow one
    ms_max, value = b.aggregate_replicas(ms_local, cells=1000, steps=10, world=world, dist=dist)
    out[rank] = (ms_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms_max, value = res[r]
        assert ms_max == 125.0
        # 2 replicas x 1000 nodes x 10 steps in 0.125 s
        assert abs(value - 2 * 1000 * 10 / 0.125 / 1e6) < 1e-12


def test_single_process_aggregation():
    b = _bench()
    ms_max, value = b.aggregate_replicas(50.0, cells=10 ** 6, steps=100, world=1)
    assert ms_max == 50.0 and abs(value - 2000.0) < 1e-9


def test_cpu_baseline_sample_lasts_at_least_its_bound():
    """The CPU baseline repeats its oracle calls until the requested seconds
    of work are timed, and its MLUPS count every update it timed."""
    b = _bench()
    mlups, cores, seconds, done = b.cpu_baseline(8, 2, min_seconds=0.3)
    assert seconds >= 0.3 and done >= 2 and done % 2 == 0
    assert cores >= 1
    assert abs(mlups - 8 ** 3 * done / seconds / 1e6) <= 1e-9 * mlups
