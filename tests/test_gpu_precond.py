"""Preconditioned CG through the C ABI against the float64 oracle.

The oracle keeps plain CG: the solution of the destriping equation, not the path
to it, is what a preconditioner may not change.  Bars as in the parity tests:
solves within 1e-5 relative RMS and max |delta a| <= 1e-4 sigma (sigma = 1).

  * every kind set with the D^-1 preconditioner (tune "precond" 1) and the
    two-level one (2), both precisions;
  * a problem shaped like the 12-month IQU workload at a size the oracle solves
    in minutes: one IQU radiometer with a polarisation modulator, 1 s baselines,
    2% flagged samples in gaps, time-ordered operator (about one pixel per sample).
    At nside 512 a prefix of a few million samples is ill-posed (most pixels are
    crossed once), so the stand-in keeps the workload's pixels-per-sample,
    baseline length, flags and modulator at 5 Hz sampling and nside 64 over three
    days.  There the two-level preconditioner must cut the iterations by at least
    a third and keep the oracle's baselines.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_5609_gb300 as ds
from synth import ScanParams, make_problem

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
FAST_SKY = ScanParams(sidereal_day=7200.0)
IQU_SKY = ScanParams(f_samp=5.0, sidereal_day=7200.0)

CASES = [
    # kinds, nside, n_t, L, flag_frac, scan
    (("q", "u"), 32, 50_003, 97, 0.0, ScanParams()),
    (("I", "q", "u"), 16, 40_001, 50, 0.05, ScanParams()),
    (("iqu",), 8, 120_000, 64, 0.03, IQU_SKY),
    (("I",), 8, 10_007, 1, 0.0, ScanParams()),
    (("q",), 16, 20_000, 333, 0.0, FAST_SKY),
]
IDS = ["qu", "Iqu_flags", "iqu_flags", "I_L1", "q_only"]


def rel_rms(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.sqrt(np.mean(b ** 2))
    return float(np.sqrt(np.mean((a - b) ** 2)) / (den if den > 0 else 1.0))


def solve_gpu(prob, precision, precond, coarse_nside=None, warm=None):
    g = prob.to(DEV)
    plan = ds.destripe_plan(g.pix, g.c32, g.s32, g.valid, nside=prob.nside, kinds=prob.kinds,
                            baseline_len=prob.baseline_len, precision=precision)
    ds.destripe_tune(plan, "precond", precond)
    if coarse_nside:
        ds.destripe_tune(plan, "coarse_nside", coarse_nside)
    y = g.y.to(torch.float64 if precision == "fp64" else torch.float32).contiguous()
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV) if warm is None else \
        torch.from_numpy(warm).to(DEV)
    st, it, rel = ds.destripe_solve(plan, y, a, tol=1e-10, warm_start=warm is not None)
    m = torch.zeros(plan.n_c * plan.npix, dtype=torch.float64, device=DEV)
    ds.destripe_map(plan, y, a, m)
    info = ds.destripe_plan_info(plan)
    plan.close()
    return st, it, rel, a.cpu().numpy(), m.cpu().numpy(), info


def oracle_of(prob, precision):
    d = prob.numpy()
    if precision == "mixed":  # the mixed path reads float32 timelines
        d["y"] = prob.y.to(torch.float32).double().numpy()
    op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                          prob.baseline_len)
    return op, oracle.destripe(op, d["y"], tol=1e-10)


@pytest.mark.parametrize("precond", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_preconditioned_solve_matches_oracle(case, precision, precond):
    kinds, nside, n_t, L, ff, scan = case
    prob = make_problem(n_t, nside, kinds, baseline_len=L, f_knee=0.1, alpha=1.7, seed=11,
                        scan=scan, flag_frac=ff, flag_mean_len=200,
                        sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    op, ref = oracle_of(prob, precision)
    st, it, rel, a, m, info = solve_gpu(prob, precision, precond,
                                        coarse_nside=max(1, nside // 4))
    assert st == ds.DS_OK and rel < 1e-9, (st, it, rel)
    assert rel_rms(a, ref["a"]) < 1e-5
    assert np.abs(a - ref["a"]).max() < 1e-4
    assert rel_rms(m.reshape(op.n_c, -1)[:, op.mask], ref["map"][:, op.mask]) < 1e-5


def test_preconditioned_warm_start_matches_oracle():
    prob = make_problem(60_000, 16, ("I", "q", "u"), baseline_len=50, f_knee=0.1, alpha=1.7,
                        seed=12, flag_frac=0.03, flag_mean_len=200,
                        sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    op, ref = oracle_of(prob, "mixed")
    rng = np.random.default_rng(4)
    x0 = ref["a"] + 0.3 * rng.standard_normal(ref["a"].shape)
    st, it, rel, a, m, info = solve_gpu(prob, "mixed", 2, coarse_nside=4, warm=x0)
    assert st == ds.DS_OK and rel < 1e-9
    assert np.abs(a - ref["a"]).max() < 1e-4


def test_long_baselines_coarse_space_matches_oracle():
    # 8 s baselines on a slowly spinning scan: each baseline stays within one or two
    # cells, so the coarse space is built (one warp per baseline gathers its cells),
    # and the two-level preconditioner needs fewer iterations than D^-1 alone
    prob = make_problem(200_000, 16, ("I", "q", "u"), baseline_len=400, f_knee=0.1, alpha=1.7,
                        seed=13, scan=ScanParams(spin_period=600.0, sidereal_day=7200.0),
                        flag_frac=0.02, flag_mean_len=200,
                        sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    op, ref = oracle_of(prob, "mixed")
    iters = {}
    for pc in (1, 2):
        st, it, rel, a, m, info = solve_gpu(prob, "mixed", pc, coarse_nside=4)
        assert st == ds.DS_OK and rel < 1e-9, (pc, st, it, rel)
        assert rel_rms(a, ref["a"]) < 1e-5, pc
        assert np.abs(a - ref["a"]).max() < 1e-4, pc
        assert rel_rms(m.reshape(op.n_c, -1)[:, op.mask], ref["map"][:, op.mask]) < 1e-5
        iters[pc] = it
    assert iters[2] < iters[1], iters


LATTE_SHAPED = dict(n_t=3 * 86400 * 5, nside=64, kinds=("iqu",), baseline_len=5, f_knee=0.05,
                    alpha=1.5, seed=1004, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0},
                    flag_frac=0.02, flag_mean_len=50,
                    scan=ScanParams(f_samp=5.0, pol_rotation_period=600.0),
                    y_dtype=torch.float32)  # both precisions read the same values


@pytest.fixture(scope="module")
def latte_shaped():
    prob = make_problem(**LATTE_SHAPED)
    return prob, oracle_of(prob, "fp64")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_level_preconditioner_on_latte_shaped_problem(latte_shaped, precision):
    prob, (op, ref) = latte_shaped
    out = {}
    for pc in (0, 2):
        st, it, rel, a, m, info = solve_gpu(prob, precision, pc, coarse_nside=8)
        assert st == ds.DS_OK and rel < 1e-9, (pc, st, it, rel)
        if precision == "mixed":
            assert info["layout"] == 0  # about one pixel per sample: time-ordered operator
        assert rel_rms(a, ref["a"]) < 1e-5, pc
        assert np.abs(a - ref["a"]).max() < 1e-4, pc
        assert rel_rms(m.reshape(op.n_c, -1)[:, op.mask], ref["map"][:, op.mask]) < 1e-5
        out[pc] = it
    assert out[2] < 0.67 * out[0], out


def test_tiled_operator_solve_on_latte_shaped_problem(latte_shaped):
    # the time-tiled, pixel-sorted records (about one pixel per sample), with and
    # without the coarse correction, reach the oracle's baselines
    # (the coarse matrix's pixel term is summed over the long tiles' runs here)
    prob, (op, ref) = latte_shaped
    iters = {}
    for pc in (0, 2):
        g = prob.to(DEV)
        plan = ds.destripe_plan(g.pix, g.c32, g.s32, g.valid, nside=prob.nside,
                                kinds=prob.kinds, baseline_len=prob.baseline_len,
                                precision="mixed")
        ds.destripe_tune(plan, "layout", 3)
        ds.destripe_tune(plan, "precond", pc)
        ds.destripe_tune(plan, "coarse_nside", 8)
        a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
        st, it, rel = ds.destripe_solve(plan, g.y, a, tol=1e-10)
        assert ds.destripe_plan_info(plan)["layout"] == 3
        plan.close()
        assert st == ds.DS_OK and rel < 1e-9, (pc, st, it, rel)
        assert np.abs(a.cpu().numpy() - ref["a"]).max() < 1e-4, pc
        iters[pc] = it
    assert iters[2] < 0.67 * iters[0], iters
