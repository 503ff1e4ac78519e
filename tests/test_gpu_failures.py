"""Failure detection and the warm start through the C ABI (non-finite data and
bad starts are made on the host; nothing here faults the GPU).

  * a NaN or an infinity in the timelines, on a valid sample, makes destripe_solve
    report DS_ENAN and makes a batch refuse the problem at admission; the plan and
    the batch stay usable;
  * the same value on a flagged sample is never read: the result is finite and
    equals the clean one up to the order of the atomic sums;
  * a first solve of a fresh mixed plan that starts from a given guess (warm
    start) reaches the oracle's baselines: its first operator application comes
    before the pixel-major copy of the run records is joined to the plan's stream.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_5609_gb300 as ds
from synth import make_problem

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def problem(precision, flag_frac=0.0, n_t=80_000, nside=16, L=400, seed=21):
    ydt = torch.float32 if precision == "mixed" else torch.float64
    return make_problem(n_t, nside, ("q", "u"), baseline_len=L, f_knee=0.1, alpha=1.7,
                        seed=seed, flag_frac=flag_frac, flag_mean_len=300, y_dtype=ydt,
                        keep_f64_trig=False).to(DEV)


def plan_of(p, precision):
    return ds.destripe_plan(p.pix, p.c32, p.s32, p.valid, nside=p.nside, kinds=p.kinds,
                            baseline_len=p.baseline_len, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")],
                         ids=["nan", "inf", "-inf"])
def test_solve_reports_nonfinite_data(precision, bad):
    p = problem(precision)
    plan = plan_of(p, precision)
    y = p.y.clone()
    y[1, 12_345] = bad
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    with pytest.raises(ds.DestripeError) as e:
        ds.destripe_solve(plan, y, a, tol=1e-10)
    assert e.value.status == ds.DS_ENAN
    # the plan is still usable: the clean data solve
    st, it, rel = ds.destripe_solve(plan, p.y, a, tol=1e-10)
    assert st == ds.DS_OK and rel < 1e-9
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonfinite_value_on_flagged_sample_is_not_read(precision):
    p = problem(precision, flag_frac=0.05)
    flagged = torch.nonzero(p.valid == 0).flatten()
    assert flagged.numel() > 0
    plan = plan_of(p, precision)
    a0 = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st0, it0, _ = ds.destripe_solve(plan, p.y, a0, tol=1e-10)
    y = p.y.clone()
    y[0, flagged[::7]] = float("nan")
    y[1, flagged[3::7]] = float("inf")
    a1 = torch.zeros_like(a0)
    st1, it1, _ = ds.destripe_solve(plan, y, a1, tol=1e-10)
    assert st0 == st1 == ds.DS_OK
    assert bool(torch.isfinite(a1).all())
    assert float((a0 - a1).abs().max()) < 1e-6
    plan.close()


def test_batch_refuses_nonfinite_problem_and_keeps_serving():
    good = problem("mixed", seed=22)
    bad = problem("mixed", seed=23)
    y_bad = bad.y.clone()
    y_bad[0, 777] = float("nan")
    pl_good, pl_bad = plan_of(good, "mixed"), plan_of(bad, "mixed")
    batch = ds.destripe_batch_create(4)
    with pytest.raises(ds.DestripeError) as e:
        ds.destripe_batch_add(batch, pl_bad, y_bad, tol=1e-10)
    assert e.value.status == ds.DS_ENAN
    assert ds.destripe_batch_info(batch)["slots_used"] == 0
    slot = ds.destripe_batch_add(batch, pl_good, good.y, tol=1e-10)
    while ds.destripe_batch_step(batch, 8) > 0:
        pass
    a = torch.empty(pl_good.n_u, dtype=torch.float64, device=DEV)
    st, it, rel = ds.destripe_batch_retire(batch, slot, a)
    assert st == ds.DS_OK and rel < 1e-9
    # the refused plan can still be solved once its data are clean
    a2 = torch.zeros(pl_bad.n_u, dtype=torch.float64, device=DEV)
    st2, _, _ = ds.destripe_solve(pl_bad, bad.y, a2, tol=1e-10)
    assert st2 == ds.DS_OK
    batch.close()
    pl_good.close()
    pl_bad.close()


def test_warm_first_solve_of_fresh_run_length_plan():
    # few runs per sample: the plan holds run records, and its first solve builds
    # the pixel-major copy beside the right-hand side
    p = problem("mixed", n_t=300_000, nside=32, L=500, seed=24)
    plan = plan_of(p, "mixed")
    assert plan.info["layout"] == 2 and plan.info["n_runs"] > 0
    d = {k: v for k, v in p.to("cpu").numpy().items()}
    op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], p.nside, p.kinds, p.baseline_len)
    ref = oracle.destripe(op, d["y"], tol=1e-10)["a"]
    rng = np.random.default_rng(5)
    a = torch.from_numpy(ref + 0.1 * rng.standard_normal(ref.shape)).to(DEV)
    st, it, rel = ds.destripe_solve(plan, p.y, a, tol=1e-10, warm_start=True)
    assert st == ds.DS_OK and rel < 1e-9
    assert ds.destripe_plan_info(plan)["bin_order"] == 1
    assert np.abs(a.cpu().numpy() - ref).max() < 1e-4
    plan.close()
