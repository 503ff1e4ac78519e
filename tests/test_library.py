"""The C-ABI library builds, loads and exports every entry point that
include/destripe.h declares; struct layouts agree between C and the binding;
argument checks fail before any device work (CPU only)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_1309_5609_gb300 as ds

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "destripe.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(destripe_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return ds.load_library(build_if_missing=True)


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", ds.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (destripe_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_binding_covers_header():
    for n in declared_functions():
        assert n in ds._SIGS, n
        assert hasattr(ds, n), n


def test_struct_layout_matches_c():
    src = f"""
    #include <stdio.h>
    #include <stddef.h>
    #include "{HEADER}"
    int main(void) {{
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(ds_desc), offsetof(ds_desc, kinds),
             offsetof(ds_desc, baseline_len), offsetof(ds_desc, rcond_min),
             offsetof(ds_desc, stream), sizeof(ds_info), offsetof(ds_info, device_bytes),
             sizeof(ds_profile), sizeof(ds_batch_tuning), offsetof(ds_batch_tuning, rate_initial),
             offsetof(ds_info, n_runs));
      return 0;
    }}"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-o", exe, c], check=True)
        vals = list(map(int, subprocess.run([exe], capture_output=True, text=True,
                                            check=True).stdout.split()))
    exp = [ctypes.sizeof(ds.ds_desc), ds.ds_desc.kinds.offset, ds.ds_desc.baseline_len.offset,
           ds.ds_desc.rcond_min.offset, ds.ds_desc.stream.offset, ctypes.sizeof(ds.ds_info),
           ds.ds_info.device_bytes.offset, ctypes.sizeof(ds.ds_profile),
           ctypes.sizeof(ds.ds_batch_tuning), ds.ds_batch_tuning.rate_initial.offset,
           ds.ds_info.n_runs.offset]
    assert vals == exp


def test_strerror(lib):
    for s in range(9):
        assert lib.destripe_strerror(s)
    assert ds.destripe_strerror(ds.DS_EPIX) == "pixel index outside the map"


def _desc(**kw):
    d = ds._make_desc(kw.get("n_t", 100), kw.get("nside", 4), kw.get("kinds", ("q", "u")),
                      kw.get("L", 10), kw.get("precision", "fp64"), 1e-3, None)
    return d


@pytest.mark.parametrize("bad", [dict(n_t=0), dict(nside=3), dict(nside=16384), dict(L=0),
                                 dict(precision=7), dict(n_t=1 << 31)])
def test_plan_rejects_bad_descriptors_before_device_work(lib, bad):
    d = _desc(**bad)
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(256)
    st = lib.destripe_plan(ctypes.byref(d), dummy, dummy, dummy, None, ctypes.byref(h))
    assert st == ds.DS_EINVAL and not h.value


def test_plan_rejects_null_and_misaligned_pointers(lib):
    d = _desc()
    h = ctypes.c_void_p()
    assert lib.destripe_plan(ctypes.byref(d), None, None, None, None, ctypes.byref(h)) == ds.DS_EINVAL
    odd = ctypes.c_void_p(256 + 4)
    ok = ctypes.c_void_p(256)
    assert lib.destripe_plan(ctypes.byref(d), ok, odd, ok, None, ctypes.byref(h)) == ds.DS_EINVAL
    assert lib.destripe_plan(ctypes.byref(d), ok, ok, ok, None, None) == ds.DS_EINVAL


def test_null_plan_calls_are_rejected(lib):
    info = ds.ds_info()
    assert lib.destripe_plan_info(None, ctypes.byref(info)) == ds.DS_EINVAL
    assert lib.destripe_apply_A(None, None, None) == ds.DS_EINVAL
    assert lib.destripe_rhs(None, None, None) == ds.DS_EINVAL
    assert lib.destripe_gauge(None, None) == ds.DS_EINVAL
    assert lib.destripe_bin(None, None, None, None, None, None) == ds.DS_EINVAL
    assert lib.destripe_map(None, None, None, None, None, None) == ds.DS_EINVAL
    lib.destripe_destroy(None)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1309_5609_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_batch_tune_profile_and_host_entry_points_reject_null_before_device_work(lib):
    # every entry point checks its handles and pointers before touching the device
    out = ctypes.c_void_p()
    assert lib.destripe_batch_create(0, None, ctypes.byref(out)) == ds.DS_EINVAL
    assert lib.destripe_batch_create(4097, None, ctypes.byref(out)) == ds.DS_EINVAL
    assert lib.destripe_batch_create(8, None, None) == ds.DS_EINVAL
    slot = ctypes.c_int32()
    n = ctypes.c_int32()
    assert lib.destripe_batch_add(None, None, None, None, 1e-10, 0, ctypes.byref(slot)) == ds.DS_EINVAL
    assert lib.destripe_batch_step(None, 1, ctypes.byref(n)) == ds.DS_EINVAL
    assert lib.destripe_batch_slot_status(None, 0, None, None, None) == ds.DS_EINVAL
    assert lib.destripe_batch_retire(None, 0, None, None, None) == ds.DS_EINVAL
    assert lib.destripe_batch_tune(None, b"tile_samples", 8192.0) == ds.DS_EINVAL
    assert lib.destripe_batch_autotune(None, 4, None) == ds.DS_EINVAL
    assert lib.destripe_batch_info(None, None, None) == ds.DS_EINVAL
    lib.destripe_batch_destroy(None)
    assert lib.destripe_tune(None, b"bin_order", 1.0) == ds.DS_EINVAL
    assert lib.destripe_tune(None, b"rescan_rounds", 4.0) == ds.DS_EINVAL
    assert lib.destripe_profile(None, 1, None) == ds.DS_EINVAL
    d = _desc()
    it = ctypes.c_int32()
    rel = ctypes.c_double()
    assert lib.destripe_run_host(ctypes.byref(d), None, None, None, None, None, 1e-10, 10,
                                 None, None, None, None, ctypes.byref(it),
                                 ctypes.byref(rel)) == ds.DS_EINVAL
    bad = _desc(n_t=0)
    ok = ctypes.c_void_p(256)
    assert lib.destripe_run_host(ctypes.byref(bad), ok, ok, ok, None, ok, 1e-10, 10,
                                 None, None, None, None, ctypes.byref(it),
                                 ctypes.byref(rel)) == ds.DS_EINVAL
    assert lib.destripe_bin_noalloc(None, ok, ok, ok, None, ok, ok, None, None) == ds.DS_EINVAL
    assert lib.destripe_bin_noalloc(ctypes.byref(bad), ok, ok, ok, None, ok, ok, None,
                                    None) == ds.DS_EINVAL


def test_gapfill_and_spectrum_reject_bad_arguments_before_device_work(lib):
    ok = ctypes.c_void_p(256)
    d = _desc()
    assert lib.destripe_gapfill(None, ok, 100, 1, ok) == ds.DS_EINVAL
    assert lib.destripe_gapfill(ctypes.byref(d), None, 100, 1, ok) == ds.DS_EINVAL
    assert lib.destripe_gapfill(ctypes.byref(d), ok, 0, 1, ok) == ds.DS_EINVAL
    assert lib.destripe_gapfill(ctypes.byref(d), ok, 100, 1, None) == ds.DS_EINVAL
    bad = _desc(n_t=0)
    assert lib.destripe_gapfill(ctypes.byref(bad), ok, 100, 1, ok) == ds.DS_EINVAL
    assert lib.destripe_spectrum(None, ok, None, 64, 4, 50.0, None, ok) == ds.DS_EINVAL
    # the preconditioner's tune keys exist (a null plan is still refused first)
    assert lib.destripe_tune(None, b"precond", 2.0) == ds.DS_EINVAL
    assert lib.destripe_tune(None, b"coarse_nside", 8.0) == ds.DS_EINVAL


def test_sharded_entry_points_reject_bad_arguments_before_device_work(lib):
    ok = ctypes.c_void_p(256)
    d = _desc()
    out = ctypes.c_void_p()
    assert lib.destripe_plan_sharded(ctypes.byref(d), None, ok, ok, ok, None,
                                     ctypes.byref(out)) == ds.DS_EINVAL
    ex = ds.ds_exchange(ds.ALLREDUCE_FN(0), None)
    assert lib.destripe_plan_sharded(ctypes.byref(d), ctypes.byref(ex), ok, ok, ok, None,
                                     ctypes.byref(out)) == ds.DS_EINVAL
    it = ctypes.c_int32()
    rel = ctypes.c_double()
    assert lib.destripe_solve_sharded(None, ok, ok, 1e-10, 10, 0, ctypes.byref(it),
                                      ctypes.byref(rel)) == ds.DS_EINVAL
