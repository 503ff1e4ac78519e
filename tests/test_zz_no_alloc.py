"""destripe_bin_noalloc: the binned map computed without any device allocation
by the library, for callers that cannot allocate device memory when they need a
map.  Called through the C ABI and compared with the plan-based destripe_bin on
two calls in a row (different data, so the second call also shows that the
shared fixed scratch array is cleared between calls).  This file is collected
last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1309_5609_gb300 as ds
from synth import ScanParams, make_problem

pytestmark = pytest.mark.gpu


def rel_rms(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    den = np.sqrt(np.mean(b ** 2))
    return float(np.sqrt(np.mean((a - b) ** 2)) / (den if den > 0 else 1.0))


def reference(prob, y, precision):
    """Existing entry point: plan + destripe_bin (no baselines)."""
    plan = ds.destripe_plan(prob.pix, prob.c32, prob.s32, prob.valid, nside=prob.nside,
                            kinds=prob.kinds, baseline_len=prob.baseline_len,
                            precision=precision)
    m = torch.zeros(plan.n_c * plan.npix, dtype=torch.float64, device=y.device)
    h = torch.zeros(plan.npix, dtype=torch.int32, device=y.device)
    k = torch.zeros(plan.npix, dtype=torch.uint8, device=y.device)
    ds.destripe_bin(plan, y, None, m, h, k)
    torch.cuda.synchronize()
    plan.close()
    return m.cpu().numpy(), h.cpu().numpy(), k.cpu().numpy()


def call_c_abi(prob, y, precision):
    """The new entry point, called directly through ctypes."""
    lib = ds.load_library()
    dev = y.device
    n_c = len(ds.components(prob.kinds))
    npix = 12 * prob.nside ** 2
    m = torch.full((n_c * npix,), float("nan"), dtype=torch.float64, device=dev)
    h = torch.full((npix,), -1, dtype=torch.int32, device=dev)
    k = torch.full((npix,), 7, dtype=torch.uint8, device=dev)
    desc = ds._make_desc(prob.n_t, prob.nside, prob.kinds, 1, precision, 1e-3,
                         torch.cuda.current_stream(dev).cuda_stream)
    st = lib.destripe_bin_noalloc(ctypes.byref(desc), prob.pix.data_ptr(), prob.c32.data_ptr(),
                                  prob.s32.data_ptr(),
                                  None if prob.valid is None else prob.valid.data_ptr(),
                                  y.data_ptr(), m.data_ptr(), h.data_ptr(), k.data_ptr())
    torch.cuda.synchronize()
    return st, m.cpu().numpy(), h.cpu().numpy(), k.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_bin_matches_plan_bin_twice(precision):
    dev = torch.device("cuda:0")
    probs = [
        make_problem(200_003, 64, ("I", "q", "u"), baseline_len=500, seed=21,
                     flag_frac=0.03, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0}).to(dev),
        make_problem(150_000, 32, ("iqu",), baseline_len=50, seed=22,
                     scan=ScanParams(sidereal_day=7200.0)).to(dev),
    ]
    ydt = torch.float64 if precision == "fp64" else torch.float32
    for prob in probs:  # two calls in a row, different data and map sizes
        y = prob.y.to(ydt).contiguous()
        m_ref, h_ref, k_ref = reference(prob, y, precision)
        st, m, h, k = call_c_abi(prob, y, precision)
        assert st == ds.DS_OK, ds.destripe_strerror(st)
        assert np.array_equal(h, h_ref)
        assert np.array_equal(k, k_ref)
        assert rel_rms(m, m_ref) < 1e-11


def test_noalloc_rejects_maps_above_the_limit():
    dev = torch.device("cuda:0")
    prob = make_problem(1000, 128, ("q", "u"), baseline_len=50, seed=1).to(dev)
    lib = ds.load_library()
    desc = ds._make_desc(prob.n_t, 128, prob.kinds, 1, "fp64", 1e-3, None)
    m = torch.zeros(2 * 12 * 128 * 128, dtype=torch.float64, device=dev)
    st = lib.destripe_bin_noalloc(ctypes.byref(desc), prob.pix.data_ptr(), prob.c32.data_ptr(),
                                  prob.s32.data_ptr(), None, prob.y.data_ptr(), m.data_ptr(),
                                  None, None)
    assert st == ds.DS_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_bin_matches_the_oracle(precision):
    # hits and mask bit-exact, the binned map at the float64 bar of the parity tests
    import oracle
    dev = torch.device("cuda:0")
    prob = make_problem(120_001, 32, ("I", "q", "u"), baseline_len=500, seed=23, flag_frac=0.04,
                        sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0})
    ydt = torch.float64 if precision == "fp64" else torch.float32
    y = prob.y.to(ydt).contiguous()
    d = prob.numpy()
    op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                          prob.baseline_len)
    ref = oracle.bin_map(op, y.double().numpy())
    g = prob.to(dev)
    st, m, h, k = call_c_abi(g, y.to(dev), precision)
    assert st == ds.DS_OK
    assert np.array_equal(h, op.hits) and np.array_equal(k.astype(bool), op.mask)
    assert rel_rms(m.reshape(op.n_c, -1), ref) < 1e-11
