"""CPU-rank emulation of the multi-GPU design: one problem sharded in time over
gloo ranks (one rank per GPU in the design).

Each rank owns a contiguous range of baselines and their samples.  The plan
exchange is one all-reduce of the hits and pixel matrices; every operator apply
exchanges only the pixel sums (one all-reduce, the Export/Import pattern of
Sect. 4); CG's dot products are all-reduces of scalars.  Each rank's steps are
the oracle's own functions on its shard, so the test checks the decomposition:
the sharded operator and the sharded CG solve equal the single-rank oracle.
"""
import dataclasses
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from synth import ScanParams, make_problem

CASES = {
    "qu": dict(n_t=40_000, nside=16, kinds=("q", "u"), baseline_len=97, flag_frac=0.0),
    "Iqu_flags": dict(n_t=30_001, nside=16, kinds=("I", "q", "u"), baseline_len=50, flag_frac=0.05),
}


def _problem(case):
    return make_problem(seed=31, flag_mean_len=200, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0},
                        **CASES[case])


def _allreduce(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _rank(rank, world, port, case, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = _problem(case)
    d = prob.numpy()
    L, n_b, n_o = prob.baseline_len, prob.n_b, prob.n_o
    b_lo, b_hi = rank * n_b // world, (rank + 1) * n_b // world
    t_lo, t_hi = b_lo * L, min(b_hi * L, prob.n_t)
    sl = slice(t_lo, t_hi)
    valid = None if d["valid"] is None else d["valid"][sl]
    shard = oracle.make_plan(d["pix"][sl], d["c"][sl], d["s"][sl], valid, prob.nside,
                             prob.kinds, L)
    # plan exchange: hits and normal matrices summed over ranks, then the cut
    hits = _allreduce(shard.hits).round().astype(np.int64)
    M = _allreduce(shard.M)
    Minv, mask, rcond = oracle.pixel_cut(M, hits, 1e-3)
    shard = dataclasses.replace(shard, hits=hits, M=M, Minv=Minv, mask=mask, rcond=rcond,
                                v=shard.valid * mask[shard.pix])

    def apply_A(x_r):  # this rank's rows of A x, from its own baselines x_r
        z = oracle.expand(shard, x_r)
        m = oracle.pixel_solve(shard, _allreduce(oracle.pixel_sums(shard, z)))
        return oracle.baseline_sums(shard, shard.v * (z - oracle.rescan(shard, m)))

    def dot(u, v):
        return float(_allreduce(np.array([np.sum(u * v)]))[0])

    rng = np.random.default_rng(5)
    x = rng.standard_normal((n_o, n_b))
    Ax_r = apply_A(x[:, b_lo:b_hi])
    # right-hand side and CG on the shard, scalars all-reduced
    y = d["y"][:, sl]
    m_y = oracle.pixel_solve(shard, _allreduce(oracle.pixel_sums(shard, y)))
    b = oracle.baseline_sums(shard, shard.v * (y - oracle.rescan(shard, m_y)))
    a = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr, bb = dot(r, r), dot(b, b)
    it = 0
    while rr > 1e-20 * bb and it < 2000:
        q = apply_A(p)
        alpha = rr / dot(p, q)
        a += alpha * p
        r -= alpha * q
        rr_new = dot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    out[rank] = (b_lo, b_hi, Ax_r, a, it)
    dist.destroy_process_group()


@pytest.mark.parametrize("case", list(CASES))
def test_time_sharded_operator_and_solve_equal_single_rank(case):
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    port = 29521 + list(CASES).index(case)
    mp.spawn(_rank, args=(world, port, case, out), nprocs=world, join=True)
    prob = _problem(case)
    d = prob.numpy()
    plan = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                            prob.baseline_len)
    x = np.random.default_rng(5).standard_normal((prob.n_o, prob.n_b))
    ref = oracle.apply_A(plan, x).reshape(prob.n_o, prob.n_b)
    full = oracle.destripe(plan, d["y"], tol=1e-10)
    a_ref = full["a"].reshape(prob.n_o, prob.n_b)
    a_sharded = np.zeros_like(a_ref)
    for r in range(world):
        b_lo, b_hi, Ax_r, a_r, it = out[r]
        assert np.allclose(Ax_r, ref[:, b_lo:b_hi], rtol=0, atol=1e-10 * np.abs(ref).max())
        a_sharded[:, b_lo:b_hi] = a_r
    a_g = oracle.gauge(plan, a_sharded.reshape(-1)).reshape(prob.n_o, prob.n_b)
    assert np.abs(a_g - a_ref).max() < 1e-7
