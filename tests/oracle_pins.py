"""Pins of the float64 oracle against facts that the paper and the mathematics fix.

Each pin returns (ok, detail).  They are used twice: by test_oracle.py, which
requires every pin to hold, and by the planted-mistake test, which plants a
plausible error in the oracle (on the CPU) and requires at least one pin to fail.
"""
from __future__ import annotations

import json
import os
from fractions import Fraction

import numpy as np

import oracle.core as O
from oracle.dense import dense_solve, dense_system
from synth import ScanParams, make_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TINY_SCAN = ScanParams(f_samp=1.0)  # 6 deg of azimuth per sample: many crossings per pixel
# IQU needs a spread of parallactic angles per pixel: a fast-turning sky gives it
IQU_SCAN = ScanParams(f_samp=1.0, sidereal_day=7200.0)


def tiny(kinds, n_t=None, nside=4, L=40, seed=3, noise=True, signal=True, offsets=None,
         flag_frac=0.0, f64_trig=False):
    iqu = "iqu" in kinds
    if n_t is None:
        n_t = 4000 if iqu else 1200
    p = make_problem(n_t, nside, kinds, baseline_len=L, f_knee=0.05, alpha=1.7, seed=seed,
                     scan=IQU_SCAN if iqu else TINY_SCAN, noise=noise, signal=signal,
                     offsets=offsets, flag_frac=flag_frac, flag_mean_len=20)
    d = p.numpy()
    if f64_trig:
        d["c"] = p.c64.numpy()
        d["s"] = p.s64.numpy()
    d["sky"] = p.sky.numpy()
    d["problem"] = p
    return d


def plan_of(d, rcond_min=1e-3):
    return O.make_plan(d["pix"], d["c"], d["s"], d["valid"], d["nside"], d["kinds"],
                       d["baseline_len"], rcond_min)


def _frac(x):
    return float(Fraction(x))


def pin_golden(name):
    g = json.load(open(os.path.join(GOLDEN, name)))
    kinds = tuple(g["kinds"])
    y = np.array([[_frac(v) for v in row] for row in g["y"]])
    plan = O.make_plan(g["pix"], g["cos2psi"], g["sin2psi"], None, g["nside"], kinds,
                       g["baseline_len"])
    nb = plan.n_o * plan.n_b
    A = np.stack([O.apply_A(plan, e) for e in np.eye(nb)], 1)
    A_exp = np.array([[_frac(v) for v in row] for row in g["A"]])
    res = O.destripe(plan, y, tol=1e-14)
    ok = np.allclose(A, A_exp, atol=1e-13)
    ok &= np.allclose(res["b"], [_frac(v) for v in g["b"]], atol=1e-13)
    ok &= np.allclose(res["a"], [_frac(v) for v in g["a"]], atol=1e-12)
    for key, res_key in (("binned_map", "binned"), ("destriped_map", "map")):
        for comp, vals in g[key].items():
            ci = plan.comps.index(comp)
            for pix, v in vals.items():
                ok &= abs(res[res_key][ci, int(pix)] - _frac(v)) < 1e-12
    for pix, h in g["hits"].items():
        ok &= int(res["hits"][int(pix)]) == h
    return bool(ok), f"golden {name}"


def pin_hits_bruteforce():
    d = tiny(("q", "u"), flag_frac=0.1)
    plan = plan_of(d)
    h = np.zeros(plan.npix, dtype=np.int64)
    for t in range(plan.n_t):
        if d["valid"][t]:
            h[d["pix"][t]] += 1
    return bool(np.array_equal(h, plan.hits)), "hits vs loop"


def pin_qu_weight_is_hits():
    # Sect. 3: for a q+u polarimeter the weighting reduces to h^-1 (M_p = h_p I)
    d = tiny(("q", "u"), f64_trig=True, flag_frac=0.05)
    plan = plan_of(d)
    expect = plan.hits[:, None, None] * np.eye(2)[None]
    err = np.abs(plan.M - expect).max()
    return bool(err < 1e-10), f"|M - h I| = {err:.2e}"


def pin_iqu_matrix_bruteforce():
    d = tiny(("iqu",), n_t=300)
    plan = plan_of(d)
    M = np.zeros((plan.npix, 3, 3))
    for t in range(plan.n_t):
        w = np.array([1.0, d["c"][t], d["s"][t]])
        M[d["pix"][t]] += np.outer(w, w)
    err = np.abs(M - plan.M).max()
    return bool(err < 1e-12), f"|M - sum w w^T| = {err:.2e}"


def pin_rcond_2x2_closed_form():
    d = tiny(("q",), n_t=400)  # a lone q output: M_p is a general 2x2 matrix
    plan = plan_of(d)
    a, b, dd = plan.M[:, 0, 0], plan.M[:, 0, 1], plan.M[:, 1, 1]
    mid = (a + dd) / 2
    rad = np.sqrt(((a - dd) / 2) ** 2 + b ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        rc = np.where(mid + rad > 0, (mid - rad) / (mid + rad), 0.0)
    hit = plan.hits > 0
    err = np.abs(rc[hit] - plan.rcond[hit]).max()
    return bool(err < 1e-10), f"rcond err {err:.2e}"


def pin_binned_map_recovers_sky(kinds=("I", "q", "u")):
    # noiseless data bin back to the input sky on kept pixels (Sect. 3, Sect. 5)
    d = tiny(kinds, noise=False)
    plan = plan_of(d)
    m = O.bin_map(plan, d["y"])
    k = plan.mask
    err = np.abs(m[:, k] - d["sky"][:, k]).max()
    return bool(err < 1e-10 and k.sum() > 10), f"|m - sky| = {err:.2e} on {k.sum()} px"


def pin_operator_matches_dense(kinds=("I", "q", "u"), flag_frac=0.05):
    d = tiny(kinds, n_t=2000 if "iqu" in kinds else 600, flag_frac=flag_frac)
    plan = plan_of(d)
    D = dense_system(d["pix"], d["c"], d["s"], d["valid"], d["nside"], d["kinds"],
                     d["baseline_len"])
    nb = plan.n_o * plan.n_b
    A = np.stack([O.apply_A(plan, e) for e in np.eye(nb)], 1)
    err = np.abs(A - D["A"]).max()
    ok = err < 1e-10 * max(1.0, np.abs(D["A"]).max())
    ok &= bool(np.array_equal(plan.mask, D["keep"]))
    return bool(ok), f"|A - A_dense| = {err:.2e}"


def pin_symmetric_psd(kinds=("iqu",)):
    d = tiny(kinds, flag_frac=0.05)
    plan = plan_of(d, rcond_min=1e-2)
    rng = np.random.default_rng(0)
    nb = plan.n_o * plan.n_b
    x, y = rng.standard_normal(nb), rng.standard_normal(nb)
    Ax, Ay = O.apply_A(plan, x), O.apply_A(plan, y)
    sym = abs(x @ Ay - y @ Ax) / (np.abs(x) @ np.abs(Ay))
    psd = min(x @ Ax, y @ Ay) / (x @ x * plan.L)
    # projector: Z Z = Z on the timeline
    z = rng.standard_normal((plan.n_o, plan.n_t))
    Zz = O.apply_Z(plan, z)
    idem = np.abs(O.apply_Z(plan, Zz) - Zz).max()
    return bool(sym < 1e-13 and psd > -1e-13 and idem < 1e-11), f"sym {sym:.1e} psd {psd:.1e} idem {idem:.1e}"


def pin_single_pixel_closed_form():
    # I output, every sample on one pixel: A = diag(N_b) - N N^T / N_total
    n_t, L = 230, 50
    pix = np.full(n_t, 5)
    one = np.ones(n_t)
    plan = O.make_plan(pix, one, 0 * one, None, 1, ("I",), L)
    N = np.bincount(np.arange(n_t) // L).astype(float)
    A_exp = np.diag(N) - np.outer(N, N) / n_t
    A = np.stack([O.apply_A(plan, e) for e in np.eye(plan.n_b)], 1)
    err = np.abs(A - A_exp).max()
    return bool(err < 1e-12), f"single-pixel err {err:.2e}"


def pin_unique_pixels_give_zero():
    # every sample on its own pixel: the map absorbs everything, A = 0 and b = 0
    nside, n_t, L = 8, 700, 35
    rng = np.random.default_rng(1)
    pix = rng.permutation(12 * nside * nside)[:n_t]
    psi = rng.uniform(0, np.pi, n_t)
    ok = True
    for kinds in (("I",), ("q", "u")):
        plan = O.make_plan(pix, np.cos(2 * psi), np.sin(2 * psi), None, nside, kinds, L)
        x = rng.standard_normal(plan.n_o * plan.n_b)
        ok &= np.abs(O.apply_A(plan, x)).max() < 1e-12
        ok &= np.abs(O.rhs(plan, rng.standard_normal((plan.n_o, n_t)))).max() < 1e-12
    return bool(ok), "unique pixels"


def pin_solve_matches_pinv(kinds=("I", "q", "u"), flag_frac=0.05):
    d = tiny(kinds, n_t=600, flag_frac=flag_frac)
    plan = plan_of(d)
    res = O.destripe(plan, d["y"], tol=1e-13)
    a_d, b_d, D = dense_solve(d["pix"], d["c"], d["s"], d["valid"], d["nside"], d["kinds"],
                              d["baseline_len"], d["y"])
    err = np.abs(res["a"] - a_d).max() / np.abs(a_d).max()
    berr = np.abs(res["b"] - b_d).max() / np.abs(b_d).max()
    return bool(err < 1e-9 and berr < 1e-12), f"a vs pinv {err:.2e}, b {berr:.2e}"


def pin_signal_only_null_baselines(kinds=("I", "q", "u")):
    # Sect. 5: signal-only data give null baselines to machine precision.  The
    # right-hand side vanishes to rounding; the solve then only sees that rounding
    # (amplified by the smallest eigenvalues), so a gets a looser, still tiny, bound.
    d = tiny(kinds, noise=False, flag_frac=0.05)
    plan = plan_of(d)
    res = O.destripe(plan, d["y"], tol=1e-10)
    scale = np.abs(d["y"]).max()
    bmax = np.abs(res["b"]).max()
    amax = np.abs(res["a"]).max()
    ok = bmax < 1e-14 * scale * plan.L and amax < 1e-6 * scale
    return bool(ok), f"max |b| = {bmax:.2e}, max |a| = {amax:.2e}"


def pin_offsets_recovered(kinds=("I", "q", "u")):
    # y = F~ a_true + signal: the destriper returns a_true (up to the I gauge)
    d0 = tiny(kinds, noise=False)
    n_b = d0["problem"].n_b
    rng = np.random.default_rng(11)
    a_true = rng.standard_normal((len(kinds), n_b))
    d = tiny(kinds, noise=False, offsets=a_true)
    plan = plan_of(d)
    res = O.destripe(plan, d["y"], tol=1e-13)
    expect = O.gauge(plan, a_true.reshape(-1))
    err = np.abs(res["a"] - expect).max()
    merr = np.abs(res["map"][:, plan.mask] - (d["sky"][:, plan.mask]
                                              + _i_shift(plan, a_true))).max()
    return bool(err < 1e-9 and merr < 1e-9), f"|a - a_true| = {err:.2e}, map {merr:.2e}"


def _i_shift(plan, a_true):
    """Map offset implied by the gauge: the I map absorbs the removed constant."""
    shift = np.zeros((plan.n_c, 1))
    i_outs = [o for o, k in enumerate(plan.kinds) if k in ("I", "iqu")]
    if i_outs:
        has = O.baseline_has_data(plan)
        shift[plan.comps.index("I")] = a_true[i_outs][:, has].mean()
    return shift


def pin_rhs_is_A_of_offsets(kinds=("iqu",)):
    d0 = tiny(kinds, noise=False)
    rng = np.random.default_rng(12)
    a_true = rng.standard_normal((len(kinds), d0["problem"].n_b))
    d = tiny(kinds, noise=False, offsets=a_true)
    plan = plan_of(d, rcond_min=1e-2)
    b = O.rhs(plan, d["y"])
    Aa = O.apply_A(plan, a_true.reshape(-1))
    err = np.abs(b - Aa).max() / np.abs(Aa).max()
    return bool(err < 1e-11), f"|b - A a| = {err:.2e}"


def pin_null_mode_of_I(kinds=("I", "q", "u")):
    d = tiny(kinds)
    plan = plan_of(d)
    x = np.zeros((plan.n_o, plan.n_b))
    for o, k in enumerate(plan.kinds):
        if k in ("I", "iqu"):
            x[o] = 1.0
    err = np.abs(O.apply_A(plan, x.reshape(-1))).max()
    return bool(err < 1e-12), f"|A 1_I| = {err:.2e}"


def pin_flagged_samples_ignored(kinds=("q", "u")):
    d = tiny(kinds, flag_frac=0.1)
    plan = plan_of(d)
    r1 = O.destripe(plan, d["y"], tol=1e-12)
    y2 = d["y"].copy()
    y2[:, d["valid"] == 0] += 1e3
    r2 = O.destripe(plan, y2, tol=1e-12)
    err = max(np.abs(r1["a"] - r2["a"]).max(), np.abs(r1["map"] - r2["map"]).max())
    return bool(err < 1e-10), f"flag leak {err:.2e}"


ALL_PINS = [
    ("golden_I", lambda: pin_golden("hand_I_two_pixels.json")),
    ("golden_qu", lambda: pin_golden("hand_qu_two_pixels.json")),
    ("hits", pin_hits_bruteforce),
    ("qu_weight", pin_qu_weight_is_hits),
    ("iqu_matrix", pin_iqu_matrix_bruteforce),
    ("rcond", pin_rcond_2x2_closed_form),
    ("sky_Iqu", lambda: pin_binned_map_recovers_sky(("I", "q", "u"))),
    ("sky_iqu", lambda: pin_binned_map_recovers_sky(("iqu",))),
    ("dense_Iqu", lambda: pin_operator_matches_dense(("I", "q", "u"))),
    ("dense_iqu", lambda: pin_operator_matches_dense(("iqu",))),
    ("sym_psd", pin_symmetric_psd),
    ("single_pixel", pin_single_pixel_closed_form),
    ("unique_pixels", pin_unique_pixels_give_zero),
    ("pinv_Iqu", lambda: pin_solve_matches_pinv(("I", "q", "u"))),
    ("pinv_qu", lambda: pin_solve_matches_pinv(("q", "u"))),
    ("signal_only", pin_signal_only_null_baselines),
    ("offsets", pin_offsets_recovered),
    ("rhs", pin_rhs_is_A_of_offsets),
    ("null_I", pin_null_mode_of_I),
    ("flags", pin_flagged_samples_ignored),
]
