"""The float64 oracle against what the paper and the mathematics fix (CPU only),
plus planted mistakes that the pins must catch."""
import numpy as np
import pytest

import oracle.core as O
import oracle_pins as P
from synth import config_problem


@pytest.mark.parametrize("name,pin", P.ALL_PINS, ids=[n for n, _ in P.ALL_PINS])
def test_pin(name, pin):
    ok, detail = pin()
    assert ok, detail


def test_pinv_iqu_with_flags():
    ok, detail = P.pin_solve_matches_pinv(("iqu",), flag_frac=0.05)
    assert ok, detail


def test_last_partial_baseline():
    d = P.tiny(("q", "u"), n_t=1213, L=40)  # 1213 = 30 * 40 + 13
    plan = P.plan_of(d)
    assert plan.n_b == 31
    x = np.zeros((2, 31))
    x[:, -1] = 1.0
    z = O.expand(plan, x)
    assert z[:, -13:].min() == 1.0 and z[:, :-13].max() == 0.0
    ok, detail = P.pin_operator_matches_dense(("q", "u"))
    assert ok, detail


def test_float32_trig_reading_is_below_tolerance():
    # The problem's R is its float32 cos/sin arrays; solving with the exact float64
    # trig instead changes the baselines far below the 1e-5 relative-RMS bar.
    p = config_problem(1, n_t=1 << 17)
    d = p.numpy()
    r32 = O.destripe(P.plan_of(d), d["y"], tol=1e-10)
    d64 = dict(d, c=p.c64.numpy(), s=p.s64.numpy())
    r64 = O.destripe(P.plan_of(d64), d["y"], tol=1e-10)
    rel = np.sqrt(np.mean((r32["a"] - r64["a"]) ** 2) / np.mean(r64["a"] ** 2))
    assert rel < 1e-6, rel


# --- planted mistakes: each must make at least one pin fail --------------------------

def _mut_u_sign(kind, comps, c, s):
    ci = {k: i for i, k in enumerate(comps)}
    if kind == "u":
        return {ci["Q"]: s, ci["U"]: c}
    return ORIG["row_coefficients"](kind, comps, c, s)


def _mut_q_transposed(kind, comps, c, s):
    ci = {k: i for i, k in enumerate(comps)}
    if kind in ("q", "iqu"):
        w = ORIG["row_coefficients"](kind, comps, c, s)
        w[ci["Q"]], w[ci["U"]] = s, c
        return w
    return ORIG["row_coefficients"](kind, comps, c, s)


def _mut_apply_Z_no_weight(plan, z):
    return z - O.rescan(plan, O.bin_map(plan, z))


def _mut_expand_shift(plan, x):
    x = np.asarray(x, dtype=np.float64).reshape(plan.n_o, plan.n_b)
    return x[:, np.minimum((np.arange(plan.n_t) + 1) // plan.L, plan.n_b - 1)]


def _mut_hits_weight(M, hits, rcond_min):
    # the literal h^-1 weighting applied to every kind (wrong for IQU and single q)
    Minv, mask, rcond = ORIG["pixel_cut"](M, hits, rcond_min)
    n_c = M.shape[1]
    with np.errstate(divide="ignore"):
        hinv = np.where(hits > 0, 1.0 / np.maximum(hits, 1), 0.0)
    return hinv[:, None, None] * np.eye(n_c)[None] * mask[:, None, None], mask, rcond


def _mut_gauge_sign(plan, a):
    g = ORIG["gauge"](plan, a)
    return 2 * np.asarray(a).reshape(-1) * (g != 0) - g


def _mut_baseline_sums_len(plan, r):
    b = np.minimum(np.arange(plan.n_t) // (plan.L + 1), plan.n_b - 1)
    return np.stack([np.bincount(b, weights=r[o], minlength=plan.n_b) for o in range(plan.n_o)])


def _mut_rescan_swap(plan, m):
    m = np.asarray(m)[::-1]
    return ORIG["rescan"](plan, m)


def _mut_hits_unflagged(pix, valid, npix):
    return np.bincount(pix, minlength=npix).astype(np.int64)


def _mut_rcond_inverted(M, hits, rcond_min):
    Minv, mask, rcond = ORIG["pixel_cut"](M, hits, rcond_min)
    lam = np.linalg.eigvalsh(M)
    with np.errstate(divide="ignore", invalid="ignore"):
        rc = np.where(lam[:, 0] > 0, lam[:, -1] / lam[:, 0], 0.0)
    mask = (hits > 0) & (rc >= rcond_min)
    Minv = np.zeros_like(M)
    Minv[mask] = np.linalg.pinv(M[mask])
    return Minv, mask, rc


def _mut_cg_beta(plan, b, tol=1e-10, max_iter=10000, x0=None):
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    for it in range(min(max_iter, 60)):
        q = O.apply_A(plan, p)
        alpha = rr / float(p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = float(r @ r)
        p = r + (rr / max(rr_new, 1e-300)) * p  # inverted beta
        rr = rr_new
        if rr == 0:
            break
    return x, it, []


def _mut_keep_cut_samples(plan, z):
    # samples on cut pixels stay in the baseline sums (with a zero map there)
    return plan.valid * (z - O.rescan(plan, O.bin_map(plan, z)))


ORIG = {k: getattr(O, k) for k in ("row_coefficients", "pixel_cut", "gauge", "rescan")}

MUTATIONS = [
    ("u_row_sign", "row_coefficients", _mut_u_sign),
    ("q_row_transposed", "row_coefficients", _mut_q_transposed),
    ("Z_without_V", "apply_Z", _mut_apply_Z_no_weight),
    ("expand_off_by_one", "expand", _mut_expand_shift),
    ("literal_h_inverse", "pixel_cut", _mut_hits_weight),
    ("gauge_sign", "gauge", _mut_gauge_sign),
    ("baseline_length", "baseline_sums", _mut_baseline_sums_len),
    ("rescan_component_swap", "rescan", _mut_rescan_swap),
    ("hits_ignore_flags", "hitmap", _mut_hits_unflagged),
    ("rcond_inverted", "pixel_cut", _mut_rcond_inverted),
    ("cg_beta_inverted", "cg", _mut_cg_beta),
    ("baselines_keep_cut_samples", "apply_Z", _mut_keep_cut_samples),
]


@pytest.mark.parametrize("name,attr,fn", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, attr, fn):
    monkeypatch.setattr(O, attr, fn)
    failed = []
    for pin_name, pin in P.ALL_PINS + [("pinv_iqu", lambda: P.pin_solve_matches_pinv(("iqu",)))]:
        try:
            ok, _ = pin()
        except Exception:
            ok = False
        if not ok:
            failed.append(pin_name)
    assert failed, f"planted mistake {name} passed every pin"
