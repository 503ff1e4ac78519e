"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (mixed-precision plan, default knobs): the B-Machine-like workload (1.3e8
samples) and the LATTE-like one (1.6e9 samples).

The oracle cannot solve these sizes in seconds, but it computes sampled outputs
exactly: the operator on one baseline depends only on the pixels its samples
touch, and a pixel's normal matrix, cut and map depend only on the samples on
that pixel.  So for a few sampled baselines the test takes every sample of the
pixels they touch, renumbers those pixels, and runs the oracle on that subset:
hits and mask (bit-exact), binned and destriped maps at those pixels, and
(A x) on the sampled baselines.  The solve itself is checked through a property
that holds at any size: its residual, recomputed by an independent float64 plan.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1309_5609_gb300 as ds
from synth import config_problem

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def subset(prob, baselines):
    """Every sample on a pixel touched by the sampled baselines, pixels renumbered."""
    L, n_t = prob.baseline_len, prob.n_t
    T = torch.cat([torch.arange(b * L, min((b + 1) * L, n_t), device=DEV) for b in baselines])
    P = torch.unique(prob.pix[T])
    U = torch.nonzero(torch.isin(prob.pix, P)).squeeze(1)
    P_h, U_h = P.cpu().numpy(), U.cpu().numpy()
    local = np.searchsorted(P_h, prob.pix[U].cpu().numpy())
    valid = None if prob.valid is None else prob.valid[U].cpu().numpy()
    sub = oracle.make_plan(local, prob.c32[U].double().cpu().numpy(),
                           prob.s32[U].double().cpu().numpy(), valid, prob.nside, prob.kinds, L,
                           npix=len(P_h))
    y = prob.y[:, U].double().cpu().numpy()
    return sub, P_h, U_h, T.cpu().numpy(), y


def sampled_Ax(sub, U, T, x, L, baselines):
    """Oracle (A x) on the sampled baselines: Z applied to F~ x on the subset, summed
    over each sampled baseline's samples."""
    z = x[:, U // L]
    Zz = oracle.apply_Z(sub, z)
    pos = np.searchsorted(U, T)
    out = np.zeros((x.shape[0], len(baselines)))
    idx = {b: i for i, b in enumerate(baselines)}
    col = np.array([idx[t // L] for t in T])
    for o in range(x.shape[0]):
        out[o] = np.bincount(col, weights=Zz[o, pos], minlength=len(baselines))
    return out


def rel(a, b):
    a, b = np.asarray(a, float).ravel(), np.asarray(b, float).ravel()
    den = np.sqrt(np.mean(b ** 2))
    return float(np.sqrt(np.mean((a - b) ** 2)) / (den if den > 0 else 1.0))


@pytest.mark.parametrize("cfg", [2, 4], ids=["bmachine30d_1.3e8", "latte12m_1.6e9"])
def test_full_size_parity(cfg):
    torch.cuda.empty_cache()
    prob = config_problem(cfg, device=DEV, y_dtype=torch.float32, keep_f64_trig=False)
    n_o, n_b = prob.n_o, prob.n_b
    plan = ds.destripe_plan(prob.pix, prob.c32, prob.s32, prob.valid, nside=prob.nside,
                            kinds=prob.kinds, baseline_len=prob.baseline_len, precision="mixed")
    rng = np.random.default_rng(cfg)
    baselines = sorted(set(rng.integers(0, n_b, 12).tolist()) | {0, n_b - 1})
    sub, P, U, T, yU = subset(prob, baselines)
    cols = np.array(baselines)

    # hits, mask, binned map at the touched pixels
    m = torch.zeros(plan.n_c * plan.npix, dtype=torch.float64, device=DEV)
    hits = torch.zeros(plan.npix, dtype=torch.int32, device=DEV)
    mask = torch.zeros(plan.npix, dtype=torch.uint8, device=DEV)
    ds.destripe_bin(plan, prob.y, None, m, hits, mask)
    assert np.array_equal(hits[torch.from_numpy(P).to(DEV)].cpu().numpy(), sub.hits)
    assert np.array_equal(mask[torch.from_numpy(P).to(DEV)].cpu().numpy().astype(bool), sub.mask)
    mP = m.view(plan.n_c, plan.npix)[:, torch.from_numpy(P).to(DEV)].cpu().numpy()
    assert rel(mP, oracle.bin_map(sub, yU)) < 1e-10

    # the float32 operator on the sampled baselines
    x = torch.randn(n_o * n_b, dtype=torch.float64, device=DEV, generator=torch.Generator(DEV).manual_seed(3))
    Ax = torch.empty_like(x)
    ds.destripe_apply_A(plan, x, Ax)
    ref = sampled_Ax(sub, U, T, x.view(n_o, n_b).cpu().numpy(), prob.baseline_len, baselines)
    got = Ax.view(n_o, n_b)[:, torch.from_numpy(cols).to(DEV)].cpu().numpy()
    assert rel(got, ref) < 1e-5, rel(got, ref)
    # symmetric at full size
    x2 = torch.randn_like(x)
    Ax2 = torch.empty_like(x)
    ds.destripe_apply_A(plan, x2, Ax2)
    s12, s21 = float(torch.dot(x2, Ax)), float(torch.dot(x, Ax2))
    assert abs(s12 - s21) <= 1e-5 * max(abs(s12), 1e-300)
    del x2, Ax2

    # the solve: converged, and its residual recomputed by a float64 plan
    a = torch.zeros(n_o * n_b, dtype=torch.float64, device=DEV)
    st, iters, relres = ds.destripe_solve(plan, prob.y, a, tol=1e-10)
    assert st == ds.DS_OK, (st, iters, relres)
    assert relres < 1e-9
    # destriped map at the touched pixels, given the solved baselines
    ds.destripe_map(plan, prob.y, a, m)
    a_h = a.view(n_o, n_b).cpu().numpy()
    mref = oracle.bin_map(sub, yU - a_h[:, U // prob.baseline_len])
    mP = m.view(plan.n_c, plan.npix)[:, torch.from_numpy(P).to(DEV)].cpu().numpy()
    assert rel(mP, mref) < 1e-10
    plan.close()
    del m, Ax

    y64 = prob.y.double()
    p64 = ds.destripe_plan(prob.pix, prob.c32, prob.s32, prob.valid, nside=prob.nside,
                           kinds=prob.kinds, baseline_len=prob.baseline_len, precision="fp64")
    b = torch.empty_like(a)
    ds.destripe_rhs(p64, y64, b)
    Aa = torch.empty_like(a)
    ds.destripe_apply_A(p64, a, Aa)
    assert float(torch.linalg.norm(b - Aa) / torch.linalg.norm(b)) < 1e-8
    # the float64 operator on the sampled baselines
    ds.destripe_apply_A(p64, x, Aa)
    got = Aa.view(n_o, n_b)[:, torch.from_numpy(cols).to(DEV)].cpu().numpy()
    assert rel(got, ref) < 1e-11, rel(got, ref)
    p64.close()
    del prob, y64, a, b, Aa, x
    torch.cuda.empty_cache()
