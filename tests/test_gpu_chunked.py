"""Alternative forms of the float32 operator against the oracle and against the
time-ordered layout: the chunk-local pixel index (every chunk length, chunks
where nearly every sample has its own pixel), the run-length records, and the
time-ordered variants; every kind set, ragged tails, flagged and cut samples."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1309_5609_gb300 as ds
from synth import ScanParams, make_problem
from synth.problems import Problem

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
IQU_SKY = ScanParams(f_samp=5.0, sidereal_day=7200.0)

CASES = [
    # kinds, nside, n_t, L, flag_frac, scan
    (("q", "u"), 64, 2048 * 9 + 3, 97, 0.0, ScanParams()),
    (("I", "q", "u"), 32, 40_001, 50, 0.05, ScanParams()),
    (("iqu",), 8, 120_000, 64, 0.03, IQU_SKY),
    (("I",), 16, 10_007, 1, 0.0, ScanParams()),
    (("u", "q", "I"), 16, 30_011, 40, 0.02, ScanParams()),
]
IDS = ["qu_ragged", "Iqu_flags", "iqu_flags", "I_L1", "generic3"]


def rel_err(got, ref):
    scale = max(1e-300, float(np.sqrt(np.mean(ref ** 2))))
    return float(np.sqrt(np.mean((got - ref) ** 2))) / scale


def random_pixel_problem(n_t, nside, kinds, L, seed):
    """Every sample on an independent uniform pixel: almost no pixel repeats
    within a chunk."""
    g = torch.Generator().manual_seed(seed)
    npix = 12 * nside * nside
    pix = torch.randint(0, npix, (n_t,), generator=g, dtype=torch.int64).to(torch.int32)
    psi = torch.rand(n_t, generator=g, dtype=torch.float64) * math.pi
    c32 = torch.cos(2 * psi).float()
    s32 = torch.sin(2 * psi).float()
    y = torch.randn((len(kinds), n_t), generator=g, dtype=torch.float64)
    sky = torch.zeros((3, npix), dtype=torch.float64)
    return Problem(n_t, nside, tuple(kinds), L, pix, c32, s32, y, sky)


def check_apply(prob, chunk, layout=1, reps=2, tune=None, before=None):
    d = prob.numpy()
    op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                          prob.baseline_len)
    gp = prob.to(DEV)
    plan = ds.destripe_plan(gp.pix, gp.c32, gp.s32, gp.valid, nside=prob.nside,
                            kinds=prob.kinds, baseline_len=prob.baseline_len, precision="mixed")
    for k, v in (before or {}).items():  # keys that shape the layout's build
        ds.destripe_tune(plan, k, v)
    ds.destripe_tune(plan, "layout", layout)
    if chunk is not None:
        ds.destripe_tune(plan, "chunk", chunk)
    for k, v in (tune or {}).items():
        ds.destripe_tune(plan, k, v)
    rng = np.random.default_rng(17)
    out = []
    for _ in range(reps):  # repeated: the pixel sums must come back cleared
        x = rng.standard_normal(plan.n_u)
        Ax = torch.empty(plan.n_u, dtype=torch.float64, device=DEV)
        ds.destripe_apply_A(plan, torch.from_numpy(x).to(DEV), Ax)
        ref = oracle.apply_A(op, x)
        got = Ax.cpu().numpy()
        assert rel_err(got, ref) < 1e-5 or np.abs(ref).max() < 1e-9, rel_err(got, ref)
        out.append(got)
    plan.close()
    return out


@pytest.mark.parametrize("chunk", [2048, 4096, 8192, 16384])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_chunked_operator_parity(case, chunk):
    kinds, nside, n_t, L, ff, scan = case
    prob = make_problem(n_t, nside, kinds, baseline_len=L, seed=21, scan=scan, flag_frac=ff,
                        flag_mean_len=200, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    check_apply(prob, chunk)


@pytest.mark.parametrize("kinds", [("q", "u"), ("iqu",), ("I",)])
def test_chunked_operator_with_distinct_pixels(kinds):
    # nside 128: 196 608 pixels, so a 16384-sample chunk holds ~15 700 distinct ones
    prob = random_pixel_problem(16384 * 3 + 11, 128, kinds, 7, seed=3)
    for chunk in (2048, 16384):
        check_apply(prob, chunk)


@pytest.mark.parametrize("tune", [{"rescan_dedup": 1}, {"rescan_dedup": 0},
                                  {"samples_per_thread": 8}], ids=["dedup", "no_dedup", "spt8"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_time_ordered_operator_variants(case, tune):
    kinds, nside, n_t, L, ff, scan = case
    prob = make_problem(n_t, nside, kinds, baseline_len=L, seed=22, scan=scan, flag_frac=ff,
                        flag_mean_len=200, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    check_apply(prob, None, layout=0, tune=tune)


@pytest.mark.parametrize("bin_order", [0, 1], ids=["time_order", "pixel_major"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_run_length_operator_parity(case, bin_order):
    kinds, nside, n_t, L, ff, scan = case
    prob = make_problem(n_t, nside, kinds, baseline_len=L, seed=23, scan=scan, flag_frac=ff,
                        flag_mean_len=200, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    check_apply(prob, None, layout=2, tune={"bin_order": bin_order})


@pytest.mark.parametrize("bin_order", [0, 1], ids=["time_order", "pixel_major"])
@pytest.mark.parametrize("kinds", [("q", "u"), ("iqu",), ("I",)])
def test_run_length_operator_with_distinct_pixels(kinds, bin_order):
    # every run is a single sample
    check_apply(random_pixel_problem(50_003, 128, kinds, 7, seed=4), None, layout=2,
                tune={"bin_order": bin_order})


def test_pixel_major_binning_matches_time_order_and_reports_itself():
    # the two binning orders of the run records give the same operator (float32
    # summation order aside) and the same accurate solve; the plan reports the order
    prob = make_problem(300_000, 32, ("I", "q", "u"), baseline_len=250, seed=8, flag_frac=0.01,
                        flag_mean_len=300, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    gp = prob.to(DEV)
    out = {}
    for order in (0, 1):
        plan = ds.destripe_plan(gp.pix, gp.c32, gp.s32, gp.valid, nside=prob.nside,
                                kinds=prob.kinds, baseline_len=prob.baseline_len, precision="mixed")
        ds.destripe_tune(plan, "layout", 2)
        ds.destripe_tune(plan, "bin_order", order)
        assert ds.destripe_plan_info(plan)["bin_order"] == order
        x = torch.from_numpy(np.random.default_rng(3).standard_normal(plan.n_u)).to(DEV)
        Ax = torch.empty(plan.n_u, dtype=torch.float64, device=DEV)
        ds.destripe_apply_A(plan, x, Ax)
        a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
        st, it, rel = ds.destripe_solve(plan, gp.y.float().contiguous(), a, tol=1e-10)
        assert st == ds.DS_OK, (order, st, it, rel)
        out[order] = (Ax.cpu().numpy(), a.cpu().numpy())
        with pytest.raises(ds.DestripeError):
            ds.destripe_tune(plan, "bin_order", 2)
        plan.close()
    assert rel_err(out[1][0], out[0][0]) < 1e-6
    assert np.abs(out[1][1] - out[0][1]).max() < 1e-5 * max(1.0, np.abs(out[0][1]).max())


def test_run_length_solve_matches_oracle():
    prob = make_problem(300_000, 32, ("I", "q", "u"), baseline_len=250, seed=8, flag_frac=0.01,
                        flag_mean_len=300, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    d = prob.numpy()
    op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                          prob.baseline_len)
    ref = oracle.destripe(op, prob.y.float().double().numpy(), tol=1e-10)
    gp = prob.to(DEV)
    plan = ds.destripe_plan(gp.pix, gp.c32, gp.s32, gp.valid, nside=prob.nside, kinds=prob.kinds,
                            baseline_len=prob.baseline_len, precision="mixed")
    ds.destripe_tune(plan, "layout", 2)
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
    st, it, rel = ds.destripe_solve(plan, gp.y.float().contiguous(), a, tol=1e-10)
    plan.close()
    assert st == ds.DS_OK, (st, it, rel)
    assert np.abs(a.cpu().numpy() - ref["a"]).max() < 1e-4


def test_layouts_agree():
    prob = make_problem(100_000, 64, ("I", "q", "u"), baseline_len=300, seed=4)
    a = check_apply(prob, None, layout=1, reps=1)[0]
    b = check_apply(prob, None, layout=0, reps=1)[0]
    c = check_apply(prob, None, layout=2, reps=1)[0]
    assert rel_err(a, b) < 2e-6
    assert rel_err(c, b) < 2e-6


def test_plans_with_different_chunk_sizes_coexist():
    # the shared-memory limit of a kernel is shared by all plans: a plan built
    # after another (with smaller shared arrays) must not break the first one
    prob = make_problem(200_000, 64, ("q", "u"), baseline_len=100, seed=9)
    gp = prob.to(DEV)
    plans = []
    for chunk in (16384, 2048):
        pl = ds.destripe_plan(gp.pix, gp.c32, gp.s32, None, nside=64, kinds=("q", "u"),
                              baseline_len=100, precision="mixed")
        ds.destripe_tune(pl, "chunk", chunk)
        ds.destripe_tune(pl, "layout", 1)
        plans.append(pl)
    x = torch.randn(plans[0].n_u, dtype=torch.float64, device=DEV)
    outs = []
    for pl in plans:
        out = torch.empty_like(x)
        ds.destripe_apply_A(pl, x, out)
        outs.append(out.cpu().numpy())
        pl.close()
    assert rel_err(outs[0], outs[1]) < 2e-6


def test_chunked_solve_matches_oracle():
    prob = make_problem(300_000, 32, ("q", "u"), baseline_len=250, seed=8, flag_frac=0.01,
                        flag_mean_len=300)
    d = prob.numpy()
    op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                          prob.baseline_len)
    ref = oracle.destripe(op, prob.y.float().double().numpy(), tol=1e-10)
    gp = prob.to(DEV)
    for chunk in (2048, 8192):
        plan = ds.destripe_plan(gp.pix, gp.c32, gp.s32, gp.valid, nside=prob.nside,
                                kinds=prob.kinds, baseline_len=prob.baseline_len,
                                precision="mixed")
        ds.destripe_tune(plan, "chunk", chunk)
        a = torch.zeros(plan.n_u, dtype=torch.float64, device=DEV)
        st, it, rel = ds.destripe_solve(plan, gp.y.float().contiguous(), a, tol=1e-10)
        plan.close()
        assert st == ds.DS_OK, (st, it, rel)
        assert np.abs(a.cpu().numpy() - ref["a"]).max() < 1e-4


def test_tune_rejects_bad_chunks():
    prob = make_problem(5000, 8, ("q", "u"), baseline_len=50, seed=1)
    gp = prob.to(DEV)
    plan = ds.destripe_plan(gp.pix, gp.c32, gp.s32, None, nside=8, kinds=("q", "u"),
                            baseline_len=50, precision="mixed")
    for bad in (1000, 1024, 32768, 3000):
        with pytest.raises(ds.DestripeError) as e:
            ds.destripe_tune(plan, "chunk", bad)
        assert e.value.status == ds.DS_EINVAL
    plan.close()
    p64 = ds.destripe_plan(gp.pix, gp.c32, gp.s32, None, nside=8, kinds=("q", "u"),
                           baseline_len=50, precision="fp64")
    with pytest.raises(ds.DestripeError) as e:
        ds.destripe_tune(p64, "layout", 1)
    assert e.value.status == ds.DS_ESTATE
    p64.close()


def runs_per_pixel_problem(counts, nside, kinds, L, seed):
    """Pixel i of `counts` gets exactly counts[i] runs (2-4 samples each, random angles),
    interleaved round-robin with a filler pixel so that no two runs merge."""
    rng = np.random.default_rng(seed)
    npix = 12 * nside * nside
    pixels = rng.choice(npix - 1, size=len(counts), replace=False)
    filler = npix - 1
    seq = []
    for r in range(max(counts)):
        for p, k in zip(pixels, counts):
            if r < k:
                seq += [int(p)] * int(rng.integers(2, 5))
                seq += [filler] * int(rng.integers(1, 3))
    pix = torch.tensor(seq, dtype=torch.int32)
    n_t = pix.numel()
    psi = torch.from_numpy(rng.uniform(0, np.pi, n_t))
    y = torch.from_numpy(rng.standard_normal((len(kinds), n_t)))
    sky = torch.zeros((3, npix), dtype=torch.float64)
    return Problem(n_t, nside, tuple(kinds), L, pix, torch.cos(2 * psi).float(),
                   torch.sin(2 * psi).float(), y, sky)


@pytest.mark.parametrize("kinds", [("q", "u"), ("I", "q", "u")])
def test_pixel_major_binning_at_warp_step_boundaries(kinds):
    # the pixel-major binning walks a pixel's runs 64 at a time (two per lane):
    # pixels with 1, 31-33, 63-65 and 200 runs
    prob = runs_per_pixel_problem([1, 31, 32, 33, 63, 64, 65, 200], 8, kinds, 997, seed=12)
    check_apply(prob, None, layout=2, tune={"bin_order": 1})


# ---- time-tiled, pixel-sorted run records (layout 3) -----------------------------------

@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_tiled_operator_parity(case):
    kinds, nside, n_t, L, ff, scan = case
    prob = make_problem(n_t, nside, kinds, baseline_len=L, seed=23, scan=scan, flag_frac=ff,
                        flag_mean_len=200, y_dtype=torch.float64)
    check_apply(prob, None, layout=3)


@pytest.mark.parametrize("L", [1, 3, 50, 12_289, 30_000])
def test_tiled_operator_tile_edges(L):
    # baselines per tile: 12288 / n_o; L = 1 puts many tiles in a short problem, long
    # baselines put few runs' baselines far from the tile start, 30 000 makes one tile
    prob = make_problem(150_011, 16, ("I", "q", "u"), baseline_len=L, seed=24, flag_frac=0.02,
                        flag_mean_len=100, y_dtype=torch.float64)
    check_apply(prob, None, layout=3)


@pytest.mark.parametrize("tiles", [1, 7, 64, 0])
@pytest.mark.parametrize("case", [CASES[2], CASES[1], CASES[0]], ids=["iqu_sky", "Iqu", "qu"])
def test_tiled_binning_long_tile_lengths(case, tiles):
    # baselines per long tile of the binning: 1 (a tile per baseline), 7, 64, or the
    # default (one tile).  On the small IQU sky every pixel holds hundreds of runs
    # per tile, so pixels cross lanes, rounds of 256 records and warp chunks
    kinds, nside, n_t, L, ff, scan = case
    prob = make_problem(n_t, nside, kinds, baseline_len=L, seed=25, scan=scan, flag_frac=ff,
                        flag_mean_len=200, y_dtype=torch.float64)
    before = {"bin_tile_samples": tiles * L} if tiles else None
    check_apply(prob, None, layout=3, before=before)


def test_tiled_operator_on_random_pixels():
    # every sample on its own pixel: one run per sample, groups of one run
    prob = random_pixel_problem(200_003, 64, ("q", "u"), 25, seed=5)
    check_apply(prob, None, layout=3)
    check_apply(prob, None, layout=3, before={"bin_tile_samples": 25 * 3})


def test_tiled_rescan_fixed_point_scale_follows_the_map():
    # The rescan's fixed-point sums take their scale from the map's largest value in
    # each application: baselines scaled by 2^-100 or 2^100 (map values near 1e-30
    # and 1e30) give the operator scaled by the same factor, at the operator bar
    # against the oracle; a non-finite baseline gives non-finite output.
    kinds, nside, n_t, L, ff, scan = CASES[2]
    prob = make_problem(n_t, nside, kinds, baseline_len=L, seed=26, scan=scan, flag_frac=ff,
                        flag_mean_len=200, y_dtype=torch.float64)
    d = prob.numpy()
    op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                          prob.baseline_len)
    gp = prob.to(DEV)
    plan = ds.destripe_plan(gp.pix, gp.c32, gp.s32, gp.valid, nside=prob.nside,
                            kinds=prob.kinds, baseline_len=prob.baseline_len, precision="mixed")
    ds.destripe_tune(plan, "layout", 3)
    x = np.random.default_rng(18).standard_normal(plan.n_u)
    ref = oracle.apply_A(op, x)
    Ax = torch.empty(plan.n_u, dtype=torch.float64, device=DEV)
    for s in (2.0 ** -100, 1.0, 2.0 ** 100):
        ds.destripe_apply_A(plan, torch.from_numpy(x * s).to(DEV), Ax)
        got = Ax.cpu().numpy() / s
        assert rel_err(got, ref) < 1e-5, (s, rel_err(got, ref))
    xn = x.copy()
    xn[plan.n_u // 2] = np.nan
    ds.destripe_apply_A(plan, torch.from_numpy(xn).to(DEV), Ax)
    assert not np.isfinite(Ax.cpu().numpy()).all()
    plan.close()
