"""White-noise gap filling and timeline amplitude spectra through the C ABI
against the float64 oracle (oracle/diagnostics.py).

Bars: good samples are never written (bit-exact); filled samples within 1e-12 of
the oracle's (float64 timelines: the day statistics differ only in summation
order) or 2 float32 ulps (float32 timelines, rounded once); spectra within 1e-10
relative (float64 FFTs of the same values).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import diagnostics as dg
import paper_1309_5609_gb300 as ds
from synth import make_problem

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def problem(n_t=300_000, flag_frac=0.05, seed=31):
    return make_problem(n_t, 16, ("I", "q", "u"), baseline_len=500, f_knee=0.1, alpha=1.7,
                        seed=seed, flag_frac=flag_frac, flag_mean_len=400,
                        sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0}, y_dtype=torch.float64)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gapfill_matches_oracle(precision):
    prob = problem()
    valid = prob.valid.clone()
    valid[250_000:260_000] = 0  # with block_len 50 000 ... and one whole day below
    valid[200_000:250_000] = 0
    ydt = torch.float64 if precision == "fp64" else torch.float32
    y = prob.y.to(ydt).contiguous()
    y[:, valid == 0] = float("nan")  # what was there is never read
    ref = dg.gapfill(y.double().numpy(), valid.numpy(), 50_000, seed=2024)
    yd = y.to(DEV)
    ds.destripe_gapfill(yd, valid.to(DEV), block_len=50_000, seed=2024)
    got = yd.cpu()
    good = valid.numpy().astype(bool)
    assert torch.equal(got[:, torch.from_numpy(good)], y[:, torch.from_numpy(good)])
    g = got.double().numpy()[:, ~good]
    r = ref[:, ~good]
    assert np.isfinite(g).all()
    assert np.array_equal(g[:, (np.nonzero(~good)[0] >= 200_000) & (np.nonzero(~good)[0] < 250_000)],
                          np.zeros((3, 50_000)))
    if precision == "fp64":
        assert np.abs(g - r).max() <= 1e-12 * max(1.0, np.abs(r).max())
    else:
        ulp = np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(g - r) <= 2 * ulp)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spectra_match_oracle(precision):
    prob = problem(n_t=400_000, flag_frac=0.0, seed=32)
    g = prob.to(DEV)
    plan = ds.destripe_plan(g.pix, g.c32, g.s32, None, nside=prob.nside, kinds=prob.kinds,
                            baseline_len=prob.baseline_len, precision=precision)
    y = g.y.to(torch.float64 if precision == "fp64" else torch.float32).contiguous()
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, it, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    assert st == ds.DS_OK
    yh = y.double().cpu().numpy()
    for aa in (None, a):
        f, amp = ds.destripe_spectrum(plan, y, aa, seg_len=8192, n_bins=25, f_samp=50.0)
        z = yh if aa is None else dg.destriped_timeline(yh, aa.cpu().numpy(), prob.baseline_len)
        for o in range(plan.n_o):
            fr, ar = dg.amplitude_spectrum(z[o], 50.0, 8192, 25)
            assert np.allclose(f.cpu().numpy(), fr, rtol=1e-12)
            assert np.allclose(amp[o].cpu().numpy(), ar, rtol=1e-10, atol=0)
    plan.close()


def test_destriping_removes_low_frequency_amplitude():
    # the paper's observation (Sect. 6): below the baseline frequency the destriped
    # timeline of a 1/f channel holds far less amplitude than the raw one
    prob = make_problem(600_000, 16, ("q", "u"), baseline_len=500, f_knee=0.5, alpha=1.7,
                        seed=34, signal=False, y_dtype=torch.float64)
    g = prob.to(DEV)
    plan = ds.destripe_plan(g.pix, g.c32, g.s32, None, nside=prob.nside, kinds=prob.kinds,
                            baseline_len=prob.baseline_len, precision="fp64")
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, it, rel = ds.destripe_solve(plan, g.y, a, tol=1e-10)
    assert st == ds.DS_OK
    f, raw = ds.destripe_spectrum(plan, g.y, None, seg_len=1 << 16, n_bins=60, f_samp=50.0)
    f, dst = ds.destripe_spectrum(plan, g.y, a, seg_len=1 << 16, n_bins=60, f_samp=50.0)
    low = f.cpu().numpy() < 0.25 * 50.0 / prob.baseline_len  # well below 1 / (10 s)
    assert low.sum() >= 1
    assert np.all(dst.cpu().numpy()[:, low] < 0.5 * raw.cpu().numpy()[:, low])
    plan.close()


def test_gap_filled_timeline_destripes_with_every_sample_valid():
    prob = problem(flag_frac=0.03, seed=33)
    g = prob.to(DEV)
    y = g.y.clone()
    ds.destripe_gapfill(y, g.valid, block_len=100_000, seed=7)
    plan = ds.destripe_plan(g.pix, g.c32, g.s32, None, nside=prob.nside, kinds=prob.kinds,
                            baseline_len=prob.baseline_len, precision="fp64")
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, it, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    assert st == ds.DS_OK and rel < 1e-9
    # the same as the oracle on the filled timeline
    d = prob.numpy()
    op = oracle.make_plan(d["pix"], d["c"], d["s"], None, prob.nside, prob.kinds, prob.baseline_len)
    ref = oracle.destripe(op, y.cpu().numpy(), tol=1e-10)
    assert np.abs(a.cpu().numpy() - ref["a"]).max() < 1e-4
    plan.close()
