"""GB300 destriper: Python binding of the C ABI in include/destripe.h.

Maximum-likelihood destriping of CMB polarimeter timelines (Zonca et al. 2013,
Sect. 3): the baselines a solve [F~^T Z F~] a = F~^T Z y by conjugate gradient,
every step running in the CUDA kernels of libdestripe.so (built for sm_103a).

This module only marshals arguments: torch tensors supply device memory and
the current CUDA stream, and each function calls the C entry point of the same
name.  There is no CPU fallback: if the library cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

__all__ = [
    "DS_OK", "DS_ENOCONV", "DestripeError", "Plan", "KIND_CODE", "lib_path", "load_library",
    "destripe_plan", "destripe_plan_info", "destripe_bin", "destripe_apply_A", "destripe_rhs",
    "destripe_solve", "destripe_map", "destripe_gauge", "destripe_destroy", "destripe_strerror",
    "destripe_run_host", "destripe_profile", "destripe_bin_noalloc", "destripe_tune",
    "Batch", "destripe_batch_create", "destripe_batch_add", "destripe_batch_step",
    "destripe_batch_slot_status", "destripe_batch_retire", "destripe_batch_tune",
    "destripe_batch_info", "destripe_batch_destroy", "destripe_batch_autotune", "components",
    "destripe_gapfill", "destripe_spectrum", "destripe_plan_sharded", "destripe_solve_sharded",
    "torch_allreduce", "destripe_scan_pointing",
]

HERE = os.path.dirname(os.path.abspath(__file__))

DS_OK, DS_EINVAL, DS_ENOMEM, DS_ECUDA, DS_ENOCONV, DS_ETIMEOUT, DS_ENAN, DS_EPIX, DS_ESTATE = range(9)
DS_PREC_FP64, DS_PREC_MIXED = 0, 1
KIND_CODE = {"I": 0, "q": 1, "u": 2, "iqu": 3}
PRECISION = {"fp64": DS_PREC_FP64, "mixed": DS_PREC_MIXED}


class ds_desc(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int64), ("nside", ctypes.c_int32),
                ("n_outputs", ctypes.c_int32), ("kinds", ctypes.c_int32 * 4),
                ("baseline_len", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rcond_min", ctypes.c_double),
                ("stream", ctypes.c_void_p)]


# int32 allreduce(void* d_buf, int64 count, int32 dtype, void* stream, void* user)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_void_p, ctypes.c_void_p)
DS_DT_F64, DS_DT_F32, DS_DT_I32 = 0, 1, 2


class ds_exchange(ctypes.Structure):
    _fields_ = [("allreduce", ALLREDUCE_FN), ("user", ctypes.c_void_p)]


class ds_scan(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in (
        "f_samp", "spin_period", "elevation_deg", "latitude_deg", "az0", "lst0", "sidereal_day",
        "pol_rotation_period")]


class ds_info(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int64), ("n_baselines", ctypes.c_int64),
                ("n_unknowns", ctypes.c_int64), ("n_pix", ctypes.c_int64),
                ("n_good_pix", ctypes.c_int64), ("n_valid", ctypes.c_int64),
                ("n_outputs", ctypes.c_int32), ("n_comp", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("layout", ctypes.c_int32),
                ("bin_order", ctypes.c_int32), ("n_runs", ctypes.c_int64)]


class ds_profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("timed_iterations", ctypes.c_int64),
                ("bin_ms", ctypes.c_double), ("rescan_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("iteration_ms", ctypes.c_double)]


class ds_batch_tuning(ctypes.Structure):
    _fields_ = [("tile_samples", ctypes.c_int32), ("tile_pixels", ctypes.c_int32),
                ("tile_unknowns", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("trials", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("rate", ctypes.c_double), ("rate_initial", ctypes.c_double)]


class DestripeError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {destripe_strerror(status)} (status {status})")


_LIB = None
_LOCK = threading.Lock()

_P = ctypes.c_void_p
_SIGS = {
    "destripe_plan": (ctypes.c_int, [ctypes.POINTER(ds_desc), _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "destripe_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(ds_info)]),
    "destripe_bin": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "destripe_apply_A": (ctypes.c_int, [_P, _P, _P]),
    "destripe_rhs": (ctypes.c_int, [_P, _P, _P]),
    "destripe_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_double)]),
    "destripe_map": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "destripe_gauge": (ctypes.c_int, [_P, _P]),
    "destripe_destroy": (None, [_P]),
    "destripe_profile": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ds_profile)]),
    "destripe_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "destripe_tune": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_double]),
    "destripe_batch_create": (ctypes.c_int, [ctypes.c_int32, _P, ctypes.POINTER(_P)]),
    "destripe_batch_add": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32)]),
    "destripe_batch_step": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "destripe_batch_slot_status": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                                  ctypes.POINTER(ctypes.c_int32),
                                                  ctypes.POINTER(ctypes.c_double)]),
    "destripe_batch_retire": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_double)]),
    "destripe_batch_tune": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_double]),
    "destripe_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "destripe_batch_destroy": (None, [_P]),
    "destripe_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ds_batch_tuning)]),
    "destripe_bin_noalloc": (ctypes.c_int, [ctypes.POINTER(ds_desc), _P, _P, _P, _P, _P, _P, _P,
                                            _P]),
    "destripe_scan_pointing": (ctypes.c_int, [ctypes.POINTER(ds_scan), ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P]),
    "destripe_plan_sharded": (ctypes.c_int, [ctypes.POINTER(ds_desc), ctypes.POINTER(ds_exchange),
                                             _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "destripe_solve_sharded": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_double)]),
    "destripe_gapfill": (ctypes.c_int, [ctypes.POINTER(ds_desc), _P, ctypes.c_int64,
                                        ctypes.c_uint64, _P]),
    "destripe_spectrum": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_double, _P, _P]),
    "destripe_run_host": (ctypes.c_int, [ctypes.POINTER(ds_desc), _P, _P, _P, _P, _P,
                                         ctypes.c_double, ctypes.c_int32, _P, _P, _P, _P,
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double)]),
}


def lib_path() -> str:
    return os.path.join(HERE, "libdestripe.so")


def load_library(build_if_missing: bool = True):
    """Load libdestripe.so (building it with nvcc if it is missing or stale)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if build_if_missing:
            from . import build as _build
            _build.build()
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"destriper library not built: {path} is missing")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
        return lib


def destripe_strerror(status: int) -> str:
    try:
        return load_library(build_if_missing=False).destripe_strerror(int(status)).decode()
    except Exception:
        return f"status {status}"


def components(kinds: Sequence[str]) -> tuple:
    has_i = any(k in ("I", "iqu") for k in kinds)
    has_p = any(k in ("q", "u", "iqu") for k in kinds)
    return ("I", "Q", "U") if has_i and has_p else (("Q", "U") if has_p else ("I",))


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _check(t, dtype, numel, name, device=None):
    import torch
    if t is None:
        raise ValueError(f"{name} is required")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, plan is on {device}")
    return t


class Plan:
    """Handle of a C plan plus the tensors it references (kept alive here)."""

    def __init__(self, handle, desc: ds_desc, kinds, nside, refs, device):
        self.handle = handle
        self.desc = desc
        self.kinds = tuple(kinds)
        self.nside = nside
        self._refs = refs
        self.device = device
        info = destripe_plan_info(self)
        self.n_t = info["n_samples"]
        self.n_b = info["n_baselines"]
        self.n_u = info["n_unknowns"]
        self.npix = info["n_pix"]
        self.n_c = info["n_comp"]
        self.n_o = info["n_outputs"]
        self.info = info

    @property
    def precision(self) -> str:
        return "fp64" if self.desc.precision == DS_PREC_FP64 else "mixed"

    @property
    def y_dtype(self):
        import torch
        return torch.float64 if self.desc.precision == DS_PREC_FP64 else torch.float32

    def close(self):
        if self.handle:
            load_library().destripe_destroy(self.handle)
            self.handle = None
            self._refs = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_desc(n_t, nside, kinds, baseline_len, precision, rcond_min, stream) -> ds_desc:
    d = ds_desc()
    d.n_samples = int(n_t)
    d.nside = int(nside)
    d.n_outputs = len(kinds)
    if not 1 <= len(kinds) <= 4:
        raise ValueError("1 to 4 outputs")
    for i, k in enumerate(kinds):
        d.kinds[i] = KIND_CODE[k]
    d.baseline_len = int(baseline_len)
    d.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    d.reserved = 0
    d.rcond_min = float(rcond_min)
    d.stream = stream
    return d


def destripe_plan(pix, cos2psi, sin2psi, valid=None, *, nside: int, kinds=("q", "u"),
                  baseline_len: int, precision="mixed", rcond_min: float = 1e-3,
                  stream=None) -> Plan:
    """Plan on the pointing (device tensors): int32 pix, float32 cos/sin 2psi, uint8 valid."""
    import torch
    lib = load_library()
    n_t = pix.numel()
    dev = pix.device
    _check(pix, torch.int32, n_t, "pix")
    _check(cos2psi, torch.float32, n_t, "cos2psi", dev)
    _check(sin2psi, torch.float32, n_t, "sin2psi", dev)
    if valid is not None:
        _check(valid, torch.uint8, n_t, "valid", dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    desc = _make_desc(n_t, nside, kinds, baseline_len, precision, rcond_min, stream)
    h = _P()
    st = lib.destripe_plan(ctypes.byref(desc), _ptr(pix), _ptr(cos2psi), _ptr(sin2psi),
                           _ptr(valid), ctypes.byref(h))
    if st != DS_OK:
        raise DestripeError(st, "destripe_plan")
    return Plan(h, desc, kinds, nside, (cos2psi, sin2psi), dev)


def destripe_plan_info(plan: Plan) -> dict:
    info = ds_info()
    st = load_library().destripe_plan_info(plan.handle, ctypes.byref(info))
    if st != DS_OK:
        raise DestripeError(st, "destripe_plan_info")
    return {f: getattr(info, f) for f, _ in ds_info._fields_}


def destripe_bin(plan: Plan, y, a, map_out, hits_out=None, mask_out=None):
    import torch
    _check(y, plan.y_dtype, plan.n_o * plan.n_t, "y", plan.device)
    if a is not None:
        _check(a, torch.float64, plan.n_u, "a", plan.device)
    _check(map_out, torch.float64, plan.n_c * plan.npix, "map", plan.device)
    if hits_out is not None:
        _check(hits_out, torch.int32, plan.npix, "hits", plan.device)
    if mask_out is not None:
        _check(mask_out, torch.uint8, plan.npix, "mask", plan.device)
    st = load_library().destripe_bin(plan.handle, _ptr(y), _ptr(a), _ptr(map_out),
                                     _ptr(hits_out), _ptr(mask_out))
    if st != DS_OK:
        raise DestripeError(st, "destripe_bin")


def destripe_map(plan: Plan, y, a, map_out, hits_out=None, mask_out=None):
    import torch
    _check(y, plan.y_dtype, plan.n_o * plan.n_t, "y", plan.device)
    _check(a, torch.float64, plan.n_u, "a", plan.device)
    _check(map_out, torch.float64, plan.n_c * plan.npix, "map", plan.device)
    st = load_library().destripe_map(plan.handle, _ptr(y), _ptr(a), _ptr(map_out),
                                     _ptr(hits_out), _ptr(mask_out))
    if st != DS_OK:
        raise DestripeError(st, "destripe_map")


def destripe_apply_A(plan: Plan, x, Ax):
    import torch
    _check(x, torch.float64, plan.n_u, "x", plan.device)
    _check(Ax, torch.float64, plan.n_u, "Ax", plan.device)
    st = load_library().destripe_apply_A(plan.handle, _ptr(x), _ptr(Ax))
    if st != DS_OK:
        raise DestripeError(st, "destripe_apply_A")


def destripe_rhs(plan: Plan, y, b):
    import torch
    _check(y, plan.y_dtype, plan.n_o * plan.n_t, "y", plan.device)
    _check(b, torch.float64, plan.n_u, "b", plan.device)
    st = load_library().destripe_rhs(plan.handle, _ptr(y), _ptr(b))
    if st != DS_OK:
        raise DestripeError(st, "destripe_rhs")


def destripe_solve(plan: Plan, y, a, tol: float = 1e-10, max_iter: int = 10000,
                   warm_start: bool = False):
    """Returns (status, iterations, float64 relative residual); raises on errors
    other than DS_ENOCONV."""
    import torch
    _check(y, plan.y_dtype, plan.n_o * plan.n_t, "y", plan.device)
    _check(a, torch.float64, plan.n_u, "a", plan.device)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = load_library().destripe_solve(plan.handle, _ptr(y), _ptr(a), float(tol), int(max_iter),
                                       1 if warm_start else 0, ctypes.byref(it), ctypes.byref(rr))
    if st not in (DS_OK, DS_ENOCONV):
        raise DestripeError(st, "destripe_solve")
    return st, it.value, rr.value


def destripe_gapfill(y, valid, *, block_len: int, seed: int, stream=None):
    """Fill the flagged samples of y ([n_o, n_t] float32 or float64 CUDA tensor, in
    place) with white noise of each day's good-sample mean and deviation."""
    import torch
    if y.dim() != 2:
        raise ValueError("y must be [n_outputs, n_samples]")
    n_o, n_t = y.shape
    _check(valid, torch.uint8, n_t, "valid", y.device)
    if y.dtype not in (torch.float32, torch.float64) or not y.is_contiguous() or not y.is_cuda:
        raise TypeError("y must be a contiguous float32 or float64 CUDA tensor")
    if stream is None:
        stream = torch.cuda.current_stream(y.device).cuda_stream
    prec = "fp64" if y.dtype == torch.float64 else "mixed"
    desc = _make_desc(n_t, 1, ("q",) * n_o, 1, prec, 0.0, stream)
    st = load_library().destripe_gapfill(ctypes.byref(desc), _ptr(valid), int(block_len),
                                         int(seed) & ((1 << 64) - 1), _ptr(y))
    if st != DS_OK:
        raise DestripeError(st, "destripe_gapfill")


def destripe_spectrum(plan: Plan, y, a, *, seg_len: int, n_bins: int, f_samp: float):
    """Binned amplitude spectra of y (a None) or y - F~ a; returns (freq [n_bins],
    amp [n_o, n_bins]) float64 CUDA tensors."""
    import torch
    _check(y, plan.y_dtype, plan.n_o * plan.n_t, "y", plan.device)
    if a is not None:
        _check(a, torch.float64, plan.n_u, "a", plan.device)
    freq = torch.empty(n_bins, dtype=torch.float64, device=plan.device)
    amp = torch.empty((plan.n_o, n_bins), dtype=torch.float64, device=plan.device)
    st = load_library().destripe_spectrum(plan.handle, _ptr(y), _ptr(a), int(seg_len),
                                          int(n_bins), float(f_samp), _ptr(freq), _ptr(amp))
    if st != DS_OK:
        raise DestripeError(st, "destripe_spectrum")
    return freq, amp


class _DeviceView:
    """A zero-copy view of count values of a device buffer (CUDA array interface)."""

    _TYPESTR = {DS_DT_F64: "<f8", DS_DT_F32: "<f4", DS_DT_I32: "<i4"}

    def __init__(self, ptr, count, dtype):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": self._TYPESTR[dtype],
                                         "data": (int(ptr), False), "version": 3}


def torch_allreduce(group=None):
    """An all-reduce (sum) over a torch.distributed group for the sharded calls:
    with the NCCL backend it is enqueued on the library's stream on the buffer
    itself; with other backends the stream is synchronised and the values are
    summed through host memory."""
    import torch
    import torch.distributed as dist

    def fn(ptr, count, dtype, stream):
        dev = torch.device("cuda", torch.cuda.current_device())
        view = torch.as_tensor(_DeviceView(ptr, count, dtype), device=dev)
        s = torch.cuda.ExternalStream(stream, device=dev) if stream else torch.cuda.default_stream(dev)
        with torch.cuda.stream(s):
            if dist.get_backend(group) == "nccl":
                dist.all_reduce(view, group=group)
            else:
                s.synchronize()
                h = view.cpu()
                dist.all_reduce(h, group=group)
                view.copy_(h)
        return 0

    return fn


def destripe_plan_sharded(pix, cos2psi, sin2psi, valid=None, *, nside: int, kinds=("q", "u"),
                          baseline_len: int, precision="mixed", allreduce, rcond_min: float = 1e-3,
                          stream=None) -> Plan:
    """Plan on this rank's time slice (starting on a baseline boundary); allreduce(ptr,
    count, dtype, stream) sums count values at a device pointer over the ranks, in
    place (torch_allreduce() gives one over torch.distributed)."""
    import torch
    lib = load_library()
    n_t = pix.numel()
    dev = pix.device
    _check(pix, torch.int32, n_t, "pix")
    _check(cos2psi, torch.float32, n_t, "cos2psi", dev)
    _check(sin2psi, torch.float32, n_t, "sin2psi", dev)
    if valid is not None:
        _check(valid, torch.uint8, n_t, "valid", dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream

    def cb(ptr, count, dtype, st, user):
        try:
            return int(allreduce(ptr, count, dtype, st) or 0)
        except Exception:
            return 1

    cfn = ALLREDUCE_FN(cb)
    ex = ds_exchange(cfn, None)
    desc = _make_desc(n_t, nside, kinds, baseline_len, precision, rcond_min, stream)
    h = _P()
    st = lib.destripe_plan_sharded(ctypes.byref(desc), ctypes.byref(ex), _ptr(pix), _ptr(cos2psi),
                                   _ptr(sin2psi), _ptr(valid), ctypes.byref(h))
    if st != DS_OK:
        raise DestripeError(st, "destripe_plan_sharded")
    # the plan calls back into cfn until destroyed: keep it alive with the plan
    return Plan(h, desc, kinds, nside, (cos2psi, sin2psi, cfn, ex), dev)


def destripe_solve_sharded(plan: Plan, y, a, tol: float = 1e-10, max_iter: int = 10000,
                           warm_start: bool = False):
    """CG over all ranks; a is this rank's slice.  Returns (status, iterations,
    relative residual); raises on errors other than DS_ENOCONV."""
    import torch
    _check(y, plan.y_dtype, plan.n_o * plan.n_t, "y", plan.device)
    _check(a, torch.float64, plan.n_u, "a", plan.device)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = load_library().destripe_solve_sharded(plan.handle, _ptr(y), _ptr(a), float(tol),
                                               int(max_iter), 1 if warm_start else 0,
                                               ctypes.byref(it), ctypes.byref(rr))
    if st not in (DS_OK, DS_ENOCONV):
        raise DestripeError(st, "destripe_solve_sharded")
    return st, it.value, rr.value


def destripe_scan_pointing(scan, first_sample: int, n_samples: int, nside: int, device=None,
                           stream=None):
    """Pointing of an analytic scan on the device: (pix int32, cos 2psi float32,
    sin 2psi float32) tensors of n_samples.  scan: an object with the ds_scan fields
    as attributes (e.g. synth.ScanParams)."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    sc = ds_scan(*(float(getattr(scan, f)) for f, _ in ds_scan._fields_))
    pix = torch.empty(n_samples, dtype=torch.int32, device=dev)
    c = torch.empty(n_samples, dtype=torch.float32, device=dev)
    s = torch.empty(n_samples, dtype=torch.float32, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    st = load_library().destripe_scan_pointing(ctypes.byref(sc), int(first_sample), int(n_samples),
                                               int(nside), _ptr(pix), _ptr(c), _ptr(s), stream)
    if st != DS_OK:
        raise DestripeError(st, "destripe_scan_pointing")
    return pix, c, s


def destripe_gauge(plan: Plan, a):
    import torch
    _check(a, torch.float64, plan.n_u, "a", plan.device)
    st = load_library().destripe_gauge(plan.handle, _ptr(a))
    if st != DS_OK:
        raise DestripeError(st, "destripe_gauge")


def destripe_destroy(plan: Plan):
    plan.close()


def destripe_tune(plan: Plan, key: str, value: float):
    """Set a tuning knob of the plan (see include/destripe.h for the keys)."""
    st = load_library().destripe_tune(plan.handle, key.encode(), float(value))
    if st != DS_OK:
        raise DestripeError(st, f"destripe_tune({key})")


def destripe_profile(plan: Plan, enable: int = -1) -> dict:
    """enable: 1 = on (resets counters), 0 = off, -1 = unchanged; returns the counters."""
    prof = ds_profile()
    st = load_library().destripe_profile(plan.handle, int(enable), ctypes.byref(prof))
    if st != DS_OK:
        raise DestripeError(st, "destripe_profile")
    return {f: getattr(prof, f) for f, _ in ds_profile._fields_}


NOALLOC_MAX_PIX = 49152  # DS_NOALLOC_MAX_PIX: largest map of destripe_bin_noalloc (nside 64)


def destripe_bin_noalloc(pix, cos2psi, sin2psi, valid, y, map_out, hits_out=None,
                         mask_out=None, *, nside: int, kinds, precision="fp64",
                         rcond_min: float = 1e-3, stream=None):
    """Binned map from the pointing and data without any device allocation by the
    library (for callers that cannot allocate device memory at that point); all
    buffers are the caller's CUDA tensors.  Maps up to NOALLOC_MAX_PIX pixels."""
    import torch
    n_t = pix.numel()
    dev = pix.device
    _check(pix, torch.int32, n_t, "pix")
    _check(cos2psi, torch.float32, n_t, "cos2psi", dev)
    _check(sin2psi, torch.float32, n_t, "sin2psi", dev)
    if valid is not None:
        _check(valid, torch.uint8, n_t, "valid", dev)
    ydt = torch.float64 if precision == "fp64" else torch.float32
    _check(y, ydt, len(kinds) * n_t, "y", dev)
    npix = 12 * nside * nside
    _check(map_out, torch.float64, len(components(kinds)) * npix, "map", dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    desc = _make_desc(n_t, nside, kinds, 1, precision, rcond_min, stream)
    st = load_library().destripe_bin_noalloc(ctypes.byref(desc), _ptr(pix), _ptr(cos2psi),
                                             _ptr(sin2psi), _ptr(valid), _ptr(y),
                                             _ptr(map_out), _ptr(hits_out), _ptr(mask_out))
    if st != DS_OK:
        raise DestripeError(st, "destripe_bin_noalloc")


def destripe_run_host(pix, cos2psi, sin2psi, valid, y, *, nside: int, kinds, baseline_len: int,
                      precision="mixed", tol: float = 1e-10, max_iter: int = 10000,
                      rcond_min: float = 1e-3, stream=None, out_a=None, out_map=None,
                      out_hits=None, out_mask=None):
    """Whole job from host (CPU) tensors; outputs are written into the given CPU
    tensors.  Returns (status, iterations, relative residual)."""
    import torch
    lib = load_library()
    for t, name in ((pix, "pix"), (cos2psi, "cos2psi"), (sin2psi, "sin2psi"), (y, "y")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    desc = _make_desc(pix.numel(), nside, kinds, baseline_len, precision, rcond_min, stream)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = lib.destripe_run_host(ctypes.byref(desc), _ptr(pix), _ptr(cos2psi), _ptr(sin2psi),
                               _ptr(valid), _ptr(y), float(tol), int(max_iter), _ptr(out_a),
                               _ptr(out_map), _ptr(out_hits), _ptr(out_mask), ctypes.byref(it),
                               ctypes.byref(rr))
    if st not in (DS_OK, DS_ENOCONV):
        raise DestripeError(st, "destripe_run_host")
    return st, it.value, rr.value


# ---- batched and served solves ---------------------------------------------------------

class Batch:
    """Handle of a C batch (continuous batching of independent solves)."""

    def __init__(self, handle, max_slots, stream):
        self.handle = handle
        self.max_slots = max_slots
        self.stream = stream
        self._slots = {}  # slot -> (plan, y, extra refs)

    def close(self):
        if self.handle:
            load_library().destripe_batch_destroy(self.handle)
            self.handle = None
            self._slots = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def destripe_batch_create(max_slots: int = 64, stream=None) -> Batch:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    h = _P()
    st = load_library().destripe_batch_create(int(max_slots), stream, ctypes.byref(h))
    if st != DS_OK:
        raise DestripeError(st, "destripe_batch_create")
    return Batch(h, max_slots, stream)


def destripe_batch_add(batch: Batch, plan: Plan, y, a0=None, tol: float = 1e-10,
                       max_iter: int = 10000) -> int:
    import torch
    _check(y, plan.y_dtype, plan.n_o * plan.n_t, "y", plan.device)
    if a0 is not None:
        _check(a0, torch.float64, plan.n_u, "a0", plan.device)
    slot = ctypes.c_int32(-1)
    st = load_library().destripe_batch_add(batch.handle, plan.handle, _ptr(y), _ptr(a0),
                                           float(tol), int(max_iter), ctypes.byref(slot))
    if st != DS_OK:
        raise DestripeError(st, "destripe_batch_add")
    batch._slots[slot.value] = (plan, y, a0)
    return slot.value


def destripe_batch_step(batch: Batch, min_iters: int = 1) -> int:
    """Run at least min_iters CG iterations of every running problem; returns how
    many problems are still running."""
    n = ctypes.c_int32(0)
    st = load_library().destripe_batch_step(batch.handle, int(min_iters), ctypes.byref(n))
    if st != DS_OK:
        raise DestripeError(st, "destripe_batch_step")
    return n.value


def destripe_batch_slot_status(batch: Batch, slot: int):
    """(done, iterations, float64 relative residual) of a slot as of the last step."""
    d, it, rr = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
    st = load_library().destripe_batch_slot_status(batch.handle, int(slot), ctypes.byref(d),
                                                   ctypes.byref(it), ctypes.byref(rr))
    if st != DS_OK:
        raise DestripeError(st, "destripe_batch_slot_status")
    return bool(d.value), it.value, rr.value


def destripe_batch_retire(batch: Batch, slot: int, a_out=None):
    """Gauge-fix and copy out a slot's baselines; frees the slot.  Returns
    (status, iterations, relative residual); raises on errors other than DS_ENOCONV."""
    import torch
    if a_out is not None:
        plan = batch._slots[slot][0]
        _check(a_out, torch.float64, plan.n_u, "a_out", plan.device)
    it, rr = ctypes.c_int32(0), ctypes.c_double(0.0)
    st = load_library().destripe_batch_retire(batch.handle, int(slot), _ptr(a_out),
                                              ctypes.byref(it), ctypes.byref(rr))
    if st not in (DS_OK, DS_ENOCONV):
        raise DestripeError(st, "destripe_batch_retire")
    batch._slots.pop(slot, None)
    return st, it.value, rr.value


def destripe_batch_tune(batch: Batch, key: str, value: float):
    st = load_library().destripe_batch_tune(batch.handle, key.encode(), float(value))
    if st != DS_OK:
        raise DestripeError(st, f"destripe_batch_tune({key})")


def destripe_batch_autotune(batch: Batch, max_trials: int = 12) -> dict:
    """Pick the batch's launch shape by timing graph replays of its own problems
    (see include/destripe.h); returns the chosen shape and the measured rates."""
    res = ds_batch_tuning()
    st = load_library().destripe_batch_autotune(batch.handle, int(max_trials), ctypes.byref(res))
    if st != DS_OK:
        raise DestripeError(st, "destripe_batch_autotune")
    return {f: getattr(res, f) for f, _ in ds_batch_tuning._fields_ if f != "pad"}


def destripe_batch_info(batch: Batch) -> dict:
    n, l = ctypes.c_int32(0), ctypes.c_int64(0)
    st = load_library().destripe_batch_info(batch.handle, ctypes.byref(n), ctypes.byref(l))
    if st != DS_OK:
        raise DestripeError(st, "destripe_batch_info")
    return {"slots_used": n.value, "kernel_launches": l.value}


def destripe_batch_destroy(batch: Batch):
    batch.close()
