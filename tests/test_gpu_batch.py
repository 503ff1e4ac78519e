"""Batched solves through the C ABI: many uneven problems in one CUDA-graph
iteration, each result the same alone and in the mix (within the parity
tolerance), continuous admission and retirement, and the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_5609_gb300 as ds
from synth import batch_configs, make_problem

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def problems(n, seed=7, n_min=1e5, n_max=1.5e6):
    out = []
    for cfg in batch_configs(n, seed=seed, n_min=n_min, n_max=n_max):
        out.append(make_problem(device=DEV, y_dtype=torch.float32, keep_f64_trig=False, **cfg))
    return out


def plan_of(prob):
    return ds.destripe_plan(prob.pix, prob.c32, prob.s32, prob.valid, nside=prob.nside,
                            kinds=prob.kinds, baseline_len=prob.baseline_len, precision="mixed")


def run_batch(probs, max_slots=None, admit_every=None):
    """Solve all problems in one batch; with admit_every=k, problems join k at a time
    while earlier ones are iterating, and finished ones are retired as they stop."""
    plans = [plan_of(p) for p in probs]
    batch = ds.destripe_batch_create(max_slots or len(probs))
    pending = list(range(len(probs)))
    slot_of, results = {}, {}
    while pending or slot_of:
        take = len(pending) if admit_every is None else min(admit_every, len(pending))
        for _ in range(take):
            if len(slot_of) >= batch.max_slots:
                break
            i = pending.pop(0)
            slot_of[i] = ds.destripe_batch_add(batch, plans[i], probs[i].y, tol=1e-10)
        ds.destripe_batch_step(batch, 8)
        for i, sl in list(slot_of.items()):
            done, it, rel = ds.destripe_batch_slot_status(batch, sl)
            if done:
                a = torch.zeros(plans[i].n_u, dtype=torch.float64, device=DEV)
                st, it, rel = ds.destripe_batch_retire(batch, sl, a)
                results[i] = (st, it, rel, a.cpu().numpy())
                del slot_of[i]
    info = ds.destripe_batch_info(batch)
    batch.close()
    for p in plans:
        p.close()
    return results, info


def test_batch_results_equal_alone_and_in_the_mix():
    probs = problems(6)
    mixed, info = run_batch(probs)
    assert info["kernel_launches"] > 0
    for i, prob in enumerate(probs):
        alone, _ = run_batch([prob])
        st_m, it_m, rel_m, a_m = mixed[i]
        st_a, it_a, rel_a, a_a = alone[0]
        assert st_m == ds.DS_OK and st_a == ds.DS_OK
        assert rel_m < 1e-9 and rel_a < 1e-9
        assert np.abs(a_m - a_a).max() < 1e-5, i
        # and the single-problem solver
        plan = plan_of(prob)
        a_s = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
        st, it, rel = ds.destripe_solve(plan, prob.y, a_s, tol=1e-10)
        assert st == ds.DS_OK
        assert np.abs(a_m - a_s.cpu().numpy()).max() < 1e-5
        plan.close()


def test_batch_matches_oracle_on_small_problems():
    probs = problems(4, seed=11, n_min=5e4, n_max=2e5)
    res, _ = run_batch(probs)
    for i, prob in enumerate(probs):
        d = prob.numpy()
        op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                              prob.baseline_len)
        ref = oracle.destripe(op, d["y"], tol=1e-10)
        st, it, rel, a = res[i]
        assert st == ds.DS_OK
        assert np.abs(a - ref["a"]).max() < 1e-4


def test_continuous_admission_and_slot_reuse():
    probs = problems(7, seed=13)
    res_all, _ = run_batch(probs)
    # 3 slots, problems join two at a time while others iterate; slots are reused
    res_cont, _ = run_batch(probs, max_slots=3, admit_every=2)
    assert sorted(res_cont) == list(range(7))
    for i in range(7):
        assert res_cont[i][0] == ds.DS_OK
        assert np.abs(res_cont[i][3] - res_all[i][3]).max() < 1e-5


def test_batch_rejects_what_it_cannot_run():
    prob = make_problem(20_000, 16, ("q", "u"), baseline_len=100, seed=1, device=DEV,
                        y_dtype=torch.float32)
    prob_i = make_problem(20_000, 16, ("I",), baseline_len=100, seed=2, device=DEV,
                          y_dtype=torch.float32)
    batch = ds.destripe_batch_create(1)
    p64 = ds.destripe_plan(prob.pix, prob.c32, prob.s32, None, nside=16, kinds=("q", "u"),
                           baseline_len=100, precision="fp64")
    with pytest.raises(ds.DestripeError) as e:
        ds.destripe_batch_add(batch, p64, prob.y.double().contiguous())
    assert e.value.status == ds.DS_ESTATE
    p1 = plan_of(prob)
    ds.destripe_batch_add(batch, p1, prob.y)
    p2 = plan_of(prob)
    with pytest.raises(ds.DestripeError) as e:  # batch full
        ds.destripe_batch_add(batch, p2, prob.y)
    assert e.value.status == ds.DS_ESTATE
    while ds.destripe_batch_step(batch, 64) > 0:
        pass
    st, it, rel = ds.destripe_batch_retire(batch, 0, None)
    assert st == ds.DS_OK
    pi = plan_of(prob_i)
    ds.destripe_batch_add(batch, pi, prob_i.y)  # empty batch takes any component count
    while ds.destripe_batch_step(batch, 64) > 0:
        pass
    assert ds.destripe_batch_retire(batch, 0, None)[0] == ds.DS_OK
    batch.close()


def test_autotune_picks_a_shape_and_keeps_results():
    probs = problems(5, seed=17)
    ref, _ = run_batch(probs)
    plans = [plan_of(p) for p in probs]
    batch = ds.destripe_batch_create(len(probs))
    slots = [ds.destripe_batch_add(batch, pl, p.y, tol=1e-10) for pl, p in zip(plans, probs)]
    res = ds.destripe_batch_autotune(batch, max_trials=6)
    assert 1 <= res["trials"] <= 6
    assert res["rate"] > 0 and res["rate"] >= res["rate_initial"]
    assert res["blocks_per_sm"] in (4, 8, 16)
    assert res["tile_samples"] in (8192, 16384, 32768, 65536)
    assert res["tile_pixels"] in (4096, 16384, 65536)
    assert res["tile_unknowns"] in (2048, 4096, 16384)
    while ds.destripe_batch_step(batch, 8) > 0:
        pass
    for i, (sl, pl) in enumerate(zip(slots, plans)):
        a = torch.zeros(pl.n_u, dtype=torch.float64, device=DEV)
        st, it, rel = ds.destripe_batch_retire(batch, sl, a)
        assert st == ds.DS_OK
        assert np.abs(a.cpu().numpy() - ref[i][3]).max() < 1e-5
    batch.close()
    for pl in plans:
        pl.close()


def test_autotune_on_an_empty_batch_does_nothing():
    batch = ds.destripe_batch_create(4)
    res = ds.destripe_batch_autotune(batch)
    assert res["trials"] == 0
    assert (res["tile_samples"], res["tile_pixels"], res["tile_unknowns"],
            res["blocks_per_sm"]) == (16384, 16384, 4096, 8)
    batch.close()


def test_batch_mixing_run_length_and_time_ordered_problems():
    # some plans use run-length records, others the time-ordered passes (one
    # forced, one with L = 1 where every sample is its own run); each result
    # equals its problem solved alone
    probs = problems(4, seed=19)
    probs.append(make_problem(150_000, 32, ("q", "u"), baseline_len=1, seed=3, device=DEV,
                              y_dtype=torch.float32, keep_f64_trig=False))
    plans = [plan_of(p) for p in probs]
    ds.destripe_tune(plans[1], "layout", 0)
    layouts = [ds.destripe_plan_info(pl)["layout"] for pl in plans]
    assert 0 in layouts and 2 in layouts
    batch = ds.destripe_batch_create(len(probs))
    slots = [ds.destripe_batch_add(batch, pl, p.y, tol=1e-10) for pl, p in zip(plans, probs)]
    while ds.destripe_batch_step(batch, 8) > 0:
        pass
    for sl, pl, p in zip(slots, plans, probs):
        a = torch.zeros(pl.n_u, dtype=torch.float64, device=DEV)
        st, it, rel = ds.destripe_batch_retire(batch, sl, a)
        assert st == ds.DS_OK, (st, it, rel)
        alone = plan_of(p)
        a1 = torch.zeros(alone.n_u, dtype=torch.float64, device=DEV)
        st1, _, _ = ds.destripe_solve(alone, p.y, a1, tol=1e-10)
        alone.close()
        assert st1 == ds.DS_OK
        assert np.abs(a.cpu().numpy() - a1.cpu().numpy()).max() < 1e-5
    batch.close()
    for pl in plans:
        pl.close()
