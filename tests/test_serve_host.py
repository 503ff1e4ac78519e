"""Host-side logic of the serving loop and of the multi-rank benchmark (CPU)."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1309_5609_gb300.serve import device_bytes, fifo_latencies, poisson_trace


def test_fifo_latency_model():
    assert fifo_latencies([0.0, 0.5, 0.6], [1.0, 1.0, 0.1]) == [1.0, 1.5, 1.5]
    assert fifo_latencies([0.0, 10.0], [1.0, 1.0]) == [1.0, 1.0]


def test_poisson_trace_is_seeded_and_in_range():
    a = poisson_trace(20.0, 50.0, seed=1, n_min=1e5, n_max=2e8)
    b = poisson_trace(20.0, 50.0, seed=1, n_min=1e5, n_max=2e8)
    assert a == b
    assert 800 < len(a) < 1200  # 20/s for 50 s
    gaps = np.diff([r["arrival"] for r in a])
    assert abs(gaps.mean() - 0.05) < 0.01
    n = np.array([r["n_t"] for r in a])
    assert n.min() >= 1e5 and n.max() <= 2e8
    L = np.array([r["baseline_len"] for r in a])
    assert L.min() >= 25 and L.max() <= 3000
    assert {r["nside"] for r in a} <= {64, 128, 256, 512}
    assert {r["kinds"] for r in a} == {("q",), ("q", "u")}


def test_device_bytes_grows_with_request():
    assert device_bytes(2_000_000, 2, 64, 500) > device_bytes(1_000_000, 2, 64, 500)
    assert device_bytes(1_000_000, 2, 64, 50) > device_bytes(1_000_000, 2, 64, 500)
    assert device_bytes(1_000_000, 2, 512, 500) > device_bytes(1_000_000, 2, 64, 500)


def _ranks(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_ms, units = 100.0 + 50.0 * rank, 1e9 * (rank + 1)
    tmax, usum = bench.reduce_over_ranks(t_ms, units, dist, torch.device("cpu"))
    out[rank] = (tmax, usum)
    dist.destroy_process_group()


def test_replica_timing_reduces_max_time_and_total_units_over_two_gloo_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    port = 29511
    mp.spawn(_ranks, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        assert out[r] == (150.0, 3e9)
