"""CUDA path vs the float64 oracle, element by element, through the C ABI.

Bars (written here, derived in the design notes):
  * hits and mask: bit-exact;
  * float64 plans: operator and right-hand side within 1e-11 relative RMS
    (rounding order only);
  * mixed plans: operator within 1e-5 relative RMS (float32 per-sample work with
    float64 partial sums), right-hand side within 1e-11 (computed in float64);
  * solves and maps (both precisions): relative RMS <= 1e-5, baselines max
    |delta a| <= 1e-4 sigma (sigma = 1).
The mixed path reads float32 timelines; its oracle is fed the same float32
values promoted to float64.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1309_5609_gb300 as ds
from synth import ScanParams, config_problem, make_problem

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
FAST_SKY = ScanParams(sidereal_day=7200.0)  # many parallactic angles per pixel (IQU)
# 5 Hz sampling under a 2-hour sky: hours of rotation in a small problem, so that
# IQU pixels pass the rcond cut and the baseline system is well posed
IQU_SKY = ScanParams(f_samp=5.0, sidereal_day=7200.0)


def rel_rms(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.sqrt(np.mean(b ** 2))
    return float(np.sqrt(np.mean((a - b) ** 2)) / (den if den > 0 else 1.0))


def oracle_plan(prob):
    d = prob.numpy()
    return oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                            prob.baseline_len), d


def gpu_plan(prob, precision):
    g = prob.to(DEV)
    plan = ds.destripe_plan(g.pix, g.c32, g.s32, g.valid, nside=prob.nside, kinds=prob.kinds,
                            baseline_len=prob.baseline_len, precision=precision)
    ydt = torch.float64 if precision == "fp64" else torch.float32
    y = g.y.to(ydt).contiguous()
    return plan, g, y


CASES = [
    # kinds, nside, n_t, L, flag_frac, scan
    (("q", "u"), 32, 50_003, 97, 0.0, ScanParams()),
    (("I", "q", "u"), 16, 40_001, 50, 0.05, ScanParams()),
    (("iqu",), 8, 120_000, 64, 0.03, IQU_SKY),
    (("I",), 8, 10_007, 1, 0.0, ScanParams()),
    (("q",), 16, 20_000, 333, 0.0, FAST_SKY),
    (("u", "q", "I"), 16, 30_011, 40, 0.02, ScanParams()),
    (("I", "iqu"), 8, 60_000, 25, 0.0, IQU_SKY),
]
# Rank-deficient problems: most IQU pixels fail the rcond cut, so some baselines
# only see pixels that nothing else constrains and the system has null modes
# beyond the I gauge.  The baselines are not unique there; what is unique is the
# residual, which the solve must drive down in float64.
DEGENERATE = [
    (("iqu",), 16, 60_000, 64, 0.03, FAST_SKY),
    (("I", "iqu"), 16, 30_000, 25, 0.0, FAST_SKY),
]
IDS = ["qu", "Iqu_flags", "iqu_flags", "I_L1", "q_only", "uqI_generic", "I_iqu_generic"]


def case_problem(case, seed=11):
    kinds, nside, n_t, L, ff, scan = case
    return make_problem(n_t, nside, kinds, baseline_len=L, f_knee=0.1, alpha=1.7, seed=seed,
                        scan=scan, flag_frac=ff, flag_mean_len=200,
                        sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_plan_and_operator_parity(case, precision):
    prob = case_problem(case)
    op, d = oracle_plan(prob)
    plan, g, y = gpu_plan(prob, precision)
    info = plan.info
    assert info["n_good_pix"] == int(op.mask.sum())
    assert info["n_valid"] == int(op.v.sum())
    # hits and mask, bit-exact
    m = torch.zeros(plan.n_c * plan.npix, dtype=torch.float64, device=DEV)
    hits = torch.zeros(plan.npix, dtype=torch.int32, device=DEV)
    mask = torch.zeros(plan.npix, dtype=torch.uint8, device=DEV)
    ds.destripe_bin(plan, y, None, m, hits, mask)
    torch.cuda.synchronize()
    assert np.array_equal(hits.cpu().numpy(), op.hits)
    assert np.array_equal(mask.cpu().numpy().astype(bool), op.mask)
    yo = y.double().cpu().numpy().reshape(plan.n_o, plan.n_t)
    mref = oracle.bin_map(op, yo)
    assert rel_rms(m.cpu().numpy(), mref) < 1e-11
    # operator on a random vector
    rng = np.random.default_rng(5)
    x = rng.standard_normal(plan.n_u)
    xd = torch.from_numpy(x).to(DEV)
    Ax = torch.empty_like(xd)
    ds.destripe_apply_A(plan, xd, Ax)
    ref = oracle.apply_A(op, x)
    err = rel_rms(Ax.cpu().numpy(), ref)
    assert err < (1e-11 if precision == "fp64" else 1e-5), err
    # right-hand side (float64 in both precisions)
    b = torch.empty_like(xd)
    ds.destripe_rhs(plan, y, b)
    bref = oracle.rhs(op, yo)
    assert rel_rms(b.cpu().numpy(), bref) < 1e-11
    plan.close()


_SOLVE_CACHE = {}


def _oracle_solution(key, prob, y_np):
    if key not in _SOLVE_CACHE:
        op, _ = oracle_plan(prob)
        _SOLVE_CACHE[key] = (op, oracle.destripe(op, y_np, tol=1e-10))
    return _SOLVE_CACHE[key]


SOLVE_CASES = {
    "cfg1_qu_nside64": lambda: config_problem(1),
    "Iqu_nside128_prefix": lambda: config_problem(2, n_t=1_500_000, nside=128),
    "iqu_nside64_flags": lambda: config_problem(4, n_t=600_000, nside=64, baseline_len=500,
                                                scan=FAST_SKY),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(SOLVE_CASES))
def test_solve_and_map_parity(name, precision):
    prob = SOLVE_CASES[name]()
    plan, g, y = gpu_plan(prob, precision)
    yo = y.double().cpu().numpy().reshape(plan.n_o, plan.n_t)
    op, ref = _oracle_solution((name, precision), prob, yo)
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    assert st == ds.DS_OK, (st, iters, rel)
    assert rel < 1e-9
    a_h = a.cpu().numpy()
    assert rel_rms(a_h, ref["a"]) < 1e-5
    assert np.abs(a_h - ref["a"]).max() < 1e-4 * 1.0
    m = torch.zeros(plan.n_c * plan.npix, dtype=torch.float64, device=DEV)
    ds.destripe_map(plan, y, a, m)
    assert rel_rms(m.cpu().numpy(), ref["map"]) < 1e-5
    bm = torch.zeros_like(m)
    ds.destripe_bin(plan, y, None, bm)
    assert rel_rms(bm.cpu().numpy(), ref["binned"]) < 1e-11
    plan.close()


def test_warm_start_from_solution_converges_immediately():
    prob = config_problem(1, n_t=1 << 18)
    plan, g, y = gpu_plan(prob, "fp64")
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-8)
    assert st == ds.DS_OK and iters > 5
    st2, iters2, rel2 = ds.destripe_solve(plan, y, a, tol=1e-8, warm_start=True)
    assert st2 == ds.DS_OK and iters2 <= 1 and rel2 < 1e-8


def test_max_iter_reports_noconv_with_best_iterate():
    prob = config_problem(1, n_t=1 << 18)
    plan, g, y = gpu_plan(prob, "mixed")
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-14, max_iter=5)
    assert st == ds.DS_ENOCONV and iters == 5 and 0 < rel < 1
    assert torch.isfinite(a).all() and float(a.abs().max()) > 0


def test_signal_only_gives_null_baselines():
    # Sect. 5: a noiseless sky gives null baselines.  The right-hand side vanishes to
    # rounding; the solve removes its component along the I offset (rounding that
    # CG cannot reduce), and a CG run relative to the rest only amplifies it
    # through the near-null modes, so the baselines are held to the parity bar
    # (1e-4 sigma).
    prob = make_problem(400_000, 64, ("I", "q", "u"), baseline_len=500, noise=False, seed=3,
                        sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    for precision in ("fp64", "mixed"):
        plan, g, y = gpu_plan(prob, precision)
        b = torch.empty(plan.n_u, dtype=torch.float64, device=DEV)
        ds.destripe_rhs(plan, y, b)
        # float64: rounding of the sums; mixed: the float32 rounding of y itself
        eps = 1e-12 if precision == "fp64" else 1e-6
        assert float(b.abs().max()) < eps * 10.0 * 500
        a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
        ds.destripe_solve(plan, y, a, tol=1e-10)
        if precision == "fp64":
            assert float(a.abs().max()) < 1e-4
        else:
            # float32 rounding of y is input noise (6e-8 relative): compare with the
            # oracle given the same float32 values
            op, _ = oracle_plan(prob)
            ref = oracle.destripe(op, y.double().cpu().numpy().reshape(plan.n_o, plan.n_t),
                                  tol=1e-10)
            assert np.abs(a.cpu().numpy() - ref["a"]).max() < 1e-4


def test_pure_offsets_recovered():
    rng = np.random.default_rng(4)
    n_t, L = 300_000, 500
    a_true = rng.standard_normal((2, -(-n_t // L)))
    prob = make_problem(n_t, 64, ("q", "u"), baseline_len=L, noise=False, offsets=a_true,
                        seed=9)
    for precision in ("fp64", "mixed"):
        plan, g, y = gpu_plan(prob, precision)
        a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
        st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-11)
        assert st == ds.DS_OK
        assert np.abs(a.cpu().numpy() - a_true.ravel()).max() < 1e-5


@pytest.mark.parametrize("n_t,L", [(1, 1), (5, 1), (7, 100), (4099, 4096), (1000, 3)])
def test_tiny_and_ragged_sizes(n_t, L):
    prob = make_problem(n_t, 1, ("I", "q", "u"), baseline_len=L, seed=n_t, scan=FAST_SKY)
    op, d = oracle_plan(prob)
    plan, g, y = gpu_plan(prob, "fp64")
    rng = np.random.default_rng(1)
    x = rng.standard_normal(plan.n_u)
    Ax = torch.empty(plan.n_u, dtype=torch.float64, device=DEV)
    ds.destripe_apply_A(plan, torch.from_numpy(x).to(DEV), Ax)
    ref = oracle.apply_A(op, x)
    assert np.allclose(Ax.cpu().numpy(), ref, atol=1e-10 * max(1.0, np.abs(ref).max()))
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    assert st == ds.DS_OK
    res = oracle.destripe(op, d["y"], tol=1e-10)
    assert np.allclose(a.cpu().numpy(), res["a"], atol=1e-7)


def test_all_samples_flagged():
    prob = make_problem(10_000, 8, ("q", "u"), baseline_len=100, seed=2)
    g = prob.to(DEV)
    valid = torch.zeros(prob.n_t, dtype=torch.uint8, device=DEV)
    plan = ds.destripe_plan(g.pix, g.c32, g.s32, valid, nside=8, kinds=("q", "u"),
                            baseline_len=100, precision="mixed")
    assert plan.info["n_valid"] == 0 and plan.info["n_good_pix"] == 0
    y = g.y.float().contiguous()
    a = torch.ones(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    assert st == ds.DS_OK and iters == 0
    assert float(a.abs().max()) == 0.0


def test_pixel_out_of_range_is_reported():
    prob = make_problem(5000, 4, ("q", "u"), baseline_len=50, seed=1)
    g = prob.to(DEV)
    pix = g.pix.clone()
    pix[1234] = 12 * 4 * 4  # one past the last pixel
    with pytest.raises(ds.DestripeError) as e:
        ds.destripe_plan(pix, g.c32, g.s32, None, nside=4, kinds=("q", "u"), baseline_len=50)
    assert e.value.status == ds.DS_EPIX
    # the same bad index on a flagged sample is ignored
    valid = torch.ones(5000, dtype=torch.uint8, device=DEV)
    valid[1234] = 0
    plan = ds.destripe_plan(pix, g.c32, g.s32, valid, nside=4, kinds=("q", "u"), baseline_len=50)
    assert plan.info["n_valid"] <= 4999


def test_wrong_dtypes_are_rejected():
    prob = make_problem(5000, 4, ("q", "u"), baseline_len=50, seed=1)
    g = prob.to(DEV)
    with pytest.raises(TypeError):
        ds.destripe_plan(g.pix.long(), g.c32, g.s32, None, nside=4, kinds=("q", "u"),
                         baseline_len=50)
    plan = ds.destripe_plan(g.pix, g.c32, g.s32, None, nside=4, kinds=("q", "u"),
                            baseline_len=50, precision="mixed")
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    with pytest.raises(TypeError):
        ds.destripe_solve(plan, g.y.double().contiguous(), a)  # mixed plans take float32 y


def test_run_host_matches_device_path():
    prob = config_problem(1, n_t=1 << 18)
    d = prob.numpy()
    op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                          prob.baseline_len)
    y32 = prob.y.float().contiguous()
    ref = oracle.destripe(op, y32.double().numpy(), tol=1e-10)
    n_b = prob.n_b
    a = torch.zeros(2 * n_b, dtype=torch.float64)
    m = torch.zeros(2 * prob.npix, dtype=torch.float64)
    hits = torch.zeros(prob.npix, dtype=torch.int32)
    mask = torch.zeros(prob.npix, dtype=torch.uint8)
    st, iters, rel = ds.destripe_run_host(prob.pix.contiguous(), prob.c32.contiguous(),
                                          prob.s32.contiguous(), None, y32, nside=prob.nside,
                                          kinds=prob.kinds, baseline_len=prob.baseline_len,
                                          precision="mixed", tol=1e-10, out_a=a, out_map=m,
                                          out_hits=hits, out_mask=mask)
    assert st == ds.DS_OK
    assert np.array_equal(hits.numpy(), op.hits)
    assert np.array_equal(mask.numpy().astype(bool), op.mask)
    assert rel_rms(a.numpy(), ref["a"]) < 1e-5
    assert rel_rms(m.numpy(), ref["map"]) < 1e-5


def test_profile_counters_time_every_iteration():
    prob = config_problem(1, n_t=1 << 18)
    for precision in ("fp64", "mixed"):
        plan, g, y = gpu_plan(prob, precision)
        ds.destripe_profile(plan, 1)
        a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
        st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
        m = torch.zeros(plan.n_c * plan.npix, dtype=torch.float64, device=DEV)
        ds.destripe_map(plan, y, a, m)
        p = ds.destripe_profile(plan, -1)
        assert st == ds.DS_OK
        assert p["iterations"] == iters == p["timed_iterations"]
        assert p["bin_ms"] > 0 and p["rescan_ms"] > 0 and p["solve_ms"] > 0
        assert p["iteration_ms"] >= p["bin_ms"] + p["rescan_ms"]
        per_iter = 10 if precision == "mixed" else 6
        assert p["kernel_launches"] >= per_iter * iters
        ds.destripe_profile(plan, 0)
        plan.close()


@pytest.mark.parametrize("accurate_df", [0, 1])
def test_mixed_accurate_passes_both_modes(accurate_df):
    # mixed plans run the right-hand side, maps and residual refreshes either in
    # double-float (float32 pairs) or in float64: both meet the float64 bars
    prob = case_problem(CASES[1])
    op, d = oracle_plan(prob)
    plan, g, y = gpu_plan(prob, "mixed")
    ds.destripe_tune(plan, "accurate_df", accurate_df)
    yo = y.double().cpu().numpy().reshape(plan.n_o, plan.n_t)
    b = torch.empty(plan.n_u, dtype=torch.float64, device=DEV)
    ds.destripe_rhs(plan, y, b)
    assert rel_rms(b.cpu().numpy(), oracle.rhs(op, yo)) < 1e-11
    rng = np.random.default_rng(8)
    a_in = torch.from_numpy(rng.standard_normal(plan.n_u)).to(DEV)
    m = torch.zeros(plan.n_c * plan.npix, dtype=torch.float64, device=DEV)
    ds.destripe_map(plan, y, a_in, m)
    mref = oracle.bin_map(op, yo - oracle.expand(op, a_in.cpu().numpy()))
    assert rel_rms(m.cpu().numpy(), mref) < 1e-11
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    ref = oracle.destripe(op, yo, tol=1e-10)
    assert st == ds.DS_OK and rel < 1e-9
    assert rel_rms(a.cpu().numpy(), ref["a"]) < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", DEGENERATE, ids=["iqu", "I_iqu"])
def test_degenerate_problems_drive_the_float64_residual_down(case, precision):
    prob = case_problem(case)
    op, d = oracle_plan(prob)
    plan, g, y = gpu_plan(prob, precision)
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    assert st == ds.DS_OK, (st, iters, rel)
    yo = y.double().cpu().numpy().reshape(plan.n_o, plan.n_t)
    b = oracle.rhs(op, yo)
    r = b - oracle.apply_A(op, a.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_solve_every_case(case, precision):
    # every kind set, flags, L = 1 .. 333: CG (with float64 residual refreshes in
    # mixed precision) reaches the oracle's baselines
    prob = case_problem(case)
    op, d = oracle_plan(prob)
    plan, g, y = gpu_plan(prob, precision)
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    assert st == ds.DS_OK, (st, iters, rel)
    yo = y.double().cpu().numpy().reshape(plan.n_o, plan.n_t)
    ref = oracle.destripe(op, yo, tol=1e-10)
    assert np.abs(a.cpu().numpy() - ref["a"]).max() < 1e-4


def test_stalled_solve_stops_early_with_best_iterate():
    # an unreachable tolerance: the recomputed residual of a mixed plan reaches its
    # rounding floor and stalls (a float64 plan's recursive residual has no floor)
    prob = case_problem(CASES[0])
    op, d = oracle_plan(prob)
    plan, g, y = gpu_plan(prob, "mixed")
    ds.destripe_tune(plan, "stall_iters", 60)
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-30, max_iter=100000)
    assert st == ds.DS_ENOCONV, st
    assert iters < 2000
    assert rel < 1e-9  # the best iterate is returned
    yo = y.double().cpu().numpy().reshape(plan.n_o, plan.n_t)
    ref = oracle.destripe(op, yo, tol=1e-10)
    assert np.abs(a.cpu().numpy() - ref["a"]).max() < 1e-4
    plan.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[4]], ids=["qu", "q_only"])
def test_accurate_start_matches_oracle(case):
    prob = case_problem(case)
    op, d = oracle_plan(prob)
    plan, g, y = gpu_plan(prob, "mixed")
    ds.destripe_tune(plan, "accurate_start", 1)
    ds.destripe_profile(plan, 1)
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    prof = ds.destripe_profile(plan, -1)
    assert st == ds.DS_OK, (st, iters, rel)
    assert prof["iterations"] == iters and prof["timed_iterations"] == 0  # accurate graph only
    yo = y.double().cpu().numpy().reshape(plan.n_o, plan.n_t)
    ref = oracle.destripe(op, yo, tol=1e-10)
    assert np.abs(a.cpu().numpy() - ref["a"]).max() < 1e-4
    plan.close()


@pytest.mark.parametrize("rounds", [1, 3, 16])
@pytest.mark.parametrize("layout", [0, 2])
@pytest.mark.parametrize("case", [CASES[1], CASES[3], CASES[6]], ids=["Iqu_flags", "I_L1", "I_iqu"])
def test_carried_rescans_every_chunk_length(case, layout, rounds):
    # the rescans keep per-lane baseline sums across rounds of a warp's chunk and
    # flush them where a baseline ends: every chunk length, baselines of 1 to 50
    # samples, flags, both operator layouts; the right-hand side, the map and the
    # solve meet the float64 bars, the float32 operator its own
    prob = case_problem(case)
    op, d = oracle_plan(prob)
    plan, g, y = gpu_plan(prob, "mixed")
    ds.destripe_tune(plan, "layout", layout)
    ds.destripe_tune(plan, "rescan_rounds", rounds)
    yo = y.double().cpu().numpy().reshape(plan.n_o, plan.n_t)
    b = torch.empty(plan.n_u, dtype=torch.float64, device=DEV)
    ds.destripe_rhs(plan, y, b)
    assert rel_rms(b.cpu().numpy(), oracle.rhs(op, yo)) < 1e-11
    rng = np.random.default_rng(9)
    x = rng.standard_normal(plan.n_u)
    Ax = torch.empty(plan.n_u, dtype=torch.float64, device=DEV)
    ds.destripe_apply_A(plan, torch.from_numpy(x).to(DEV), Ax)
    assert rel_rms(Ax.cpu().numpy(), oracle.apply_A(op, x)) < 1e-5
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, iters, rel = ds.destripe_solve(plan, y, a, tol=1e-10)
    ref = oracle.destripe(op, yo, tol=1e-10)
    assert st == ds.DS_OK and rel < 1e-9, (st, iters, rel)
    assert rel_rms(a.cpu().numpy(), ref["a"]) < 1e-5
    m = torch.zeros(plan.n_c * plan.npix, dtype=torch.float64, device=DEV)
    ds.destripe_map(plan, y, a, m)
    mref = oracle.bin_map(op, yo - oracle.expand(op, a.cpu().numpy()))
    assert rel_rms(m.cpu().numpy(), mref) < 1e-11
    plan.close()


def test_rescan_rounds_key_bounds():
    prob = case_problem(CASES[0])
    plan, g, y = gpu_plan(prob, "mixed")
    for bad in (-1, 17, 2.5):
        with pytest.raises(ds.DestripeError):
            ds.destripe_tune(plan, "rescan_rounds", bad)
    ds.destripe_tune(plan, "rescan_rounds", 0)
    plan.close()
