"""Seeded synthetic destriping problems shaped like the paper's workloads.

A problem is one polarimeter channel (or radiometer) observing a Gaussian sky
through the spin scan of `synth.scan`:

    y_o(t) = w_o(t) . m[:, p(t)] + n_o(t)            (paper Eq. destmodel)

with one row w_o per output kind (paper Sect. 3, rotation matrices R_Q, R_U):

    I   : (1)                       on component I
    q   : ( cos 2psi,  sin 2psi)    on components (Q, U)
    u   : (-sin 2psi,  cos 2psi)    on components (Q, U)
    iqu : (1, cos 2psi, sin 2psi)   on components (I, Q, U)

The rotation matrices are stored, as the paper suggests, as length-n_t arrays of
cos 2psi and sin 2psi.  They are rounded once to float32, and that float32 array
*is* the problem's R: the signal part of y is built from it (promoted to float64)
so that a noiseless timeline lies exactly in the model's range.  The exact
float64 trig is kept beside it (c64, s64) for identities that need it.

This module holds input synthesis only; nothing in it bins, solves or rescans.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import torch

from .healpix import ang2pix_ring, npix_of, check_nside
from .noise import gap_flags, one_over_f
from .scan import ScanParams, scan_pointing

KINDS = ("I", "q", "u", "iqu")
KIND_CODE = {"I": 0, "q": 1, "u": 2, "iqu": 3}


def components(kinds) -> tuple:
    """Map components solved for a set of output kinds: (I), (Q, U) or (I, Q, U)."""
    has_i = any(k in ("I", "iqu") for k in kinds)
    has_p = any(k in ("q", "u", "iqu") for k in kinds)
    if has_i and has_p:
        return ("I", "Q", "U")
    if has_p:
        return ("Q", "U")
    if has_i:
        return ("I",)
    raise ValueError(f"no output kinds given: {kinds}")


def n_baselines(n_t: int, baseline_len: int) -> int:
    return (n_t + baseline_len - 1) // baseline_len


@dataclass
class Problem:
    n_t: int
    nside: int
    kinds: tuple
    baseline_len: int
    pix: torch.Tensor  # int32 [n_t], HEALPix RING
    c32: torch.Tensor  # float32 [n_t], cos 2psi
    s32: torch.Tensor  # float32 [n_t], sin 2psi
    y: torch.Tensor  # float64 or float32 [n_o, n_t]
    sky: torch.Tensor  # float64 [n_c, n_pix]
    valid: Optional[torch.Tensor] = None  # uint8 [n_t] (1 = good) or None
    c64: Optional[torch.Tensor] = None
    s64: Optional[torch.Tensor] = None
    meta: dict = field(default_factory=dict)

    @property
    def n_o(self) -> int:
        return len(self.kinds)

    @property
    def n_b(self) -> int:
        return n_baselines(self.n_t, self.baseline_len)

    @property
    def comps(self) -> tuple:
        return components(self.kinds)

    @property
    def npix(self) -> int:
        return npix_of(self.nside)

    def to(self, device) -> "Problem":
        def mv(x):
            return None if x is None else x.to(device)
        return Problem(self.n_t, self.nside, self.kinds, self.baseline_len, mv(self.pix),
                       mv(self.c32), mv(self.s32), mv(self.y), mv(self.sky), mv(self.valid),
                       mv(self.c64), mv(self.s64), dict(self.meta))

    def numpy(self) -> dict:
        """Host float64/int copies for the CPU oracle (trig promoted from float32)."""
        def np_(x, dt=None):
            if x is None:
                return None
            a = x.detach().cpu().numpy()
            return a.astype(dt) if dt is not None else a
        return dict(pix=np_(self.pix, np.int64), c=np_(self.c32, np.float64),
                    s=np_(self.s32, np.float64), y=np_(self.y, np.float64),
                    valid=np_(self.valid, np.uint8), nside=self.nside, kinds=self.kinds,
                    baseline_len=self.baseline_len)


def _signal(kind: str, comps: tuple, sky_at: torch.Tensor, c: torch.Tensor, s: torch.Tensor):
    """Noiseless timeline of one output: its row dotted with the sky at p(t)."""
    ci = {k: i for i, k in enumerate(comps)}
    if kind == "I":
        return sky_at[ci["I"]].clone()
    q_, u_ = sky_at[ci["Q"]], sky_at[ci["U"]]
    if kind == "q":
        return q_ * c + u_ * s
    if kind == "u":
        return -q_ * s + u_ * c
    if kind == "iqu":
        return sky_at[ci["I"]] + q_ * c + u_ * s
    raise ValueError(kind)


def make_problem(n_t: int, nside: int, kinds=("q", "u"), baseline_len: int = 500,
                 f_knee: float = 0.1, alpha: float = 1.7, sigma: float = 1.0,
                 sky_sigma: Optional[dict] = None, flag_frac: float = 0.0,
                 flag_mean_len: float = 500.0, seed: int = 0,
                 scan: ScanParams = ScanParams(), first_sample: int = 0, device="cpu",
                 y_dtype=torch.float64, signal: bool = True, noise: bool = True,
                 offsets: Optional[torch.Tensor] = None, keep_f64_trig: bool = True,
                 chunk: int = 1 << 24) -> Problem:
    """Build one seeded problem; see the module docstring for the model.

    offsets, if given, is a float64 [n_o, n_b] array of baselines added as F a
    (piecewise-constant per baseline), for offset-recovery tests.
    """
    check_nside(nside)
    kinds = tuple(kinds)
    for k in kinds:
        if k not in KINDS:
            raise ValueError(f"unknown output kind {k!r}")
    comps = components(kinds)
    sky_sigma = sky_sigma or {"I": 1.0, "Q": 1.0, "U": 1.0}
    npix = npix_of(nside)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    sky = torch.stack([
        torch.randn(npix, generator=gen, dtype=torch.float64, device=device) * float(sky_sigma.get(k, 1.0))
        for k in comps])

    pix = torch.empty(n_t, dtype=torch.int32, device=device)
    c32 = torch.empty(n_t, dtype=torch.float32, device=device)
    s32 = torch.empty(n_t, dtype=torch.float32, device=device)
    c64 = torch.empty(n_t, dtype=torch.float64, device=device) if keep_f64_trig else None
    s64 = torch.empty(n_t, dtype=torch.float64, device=device) if keep_f64_trig else None
    y = torch.zeros((len(kinds), n_t), dtype=y_dtype, device=device)
    for pos in range(0, n_t, chunk):
        m = min(chunk, n_t - pos)
        theta, phi, psi = scan_pointing(m, scan, first_sample + pos, device=device)
        p = ang2pix_ring(nside, theta, phi)
        pix[pos:pos + m] = p.to(torch.int32)
        cc = torch.cos(2.0 * psi)
        ss = torch.sin(2.0 * psi)
        cf = cc.to(torch.float32)
        sf = ss.to(torch.float32)
        c32[pos:pos + m] = cf
        s32[pos:pos + m] = sf
        if keep_f64_trig:
            c64[pos:pos + m] = cc
            s64[pos:pos + m] = ss
        if signal:
            sky_at = sky[:, p]
            for o, k in enumerate(kinds):
                y[o, pos:pos + m] = _signal(k, comps, sky_at, cf.double(), sf.double()).to(y_dtype)
        del theta, phi, psi, p, cc, ss
    if noise:
        for o in range(len(kinds)):
            g = torch.Generator(device=device)
            g.manual_seed(seed * 7919 + 101 * (o + 1))
            n = one_over_f(n_t, scan.f_samp, f_knee, alpha, sigma, g, device=device)
            y[o] += n.to(y_dtype)
            del n
    if offsets is not None:
        off = torch.as_tensor(offsets, dtype=torch.float64, device=device)
        b = torch.arange(n_t, device=device) // baseline_len
        for o in range(len(kinds)):
            y[o] += off[o, b].to(y_dtype)
    valid = None
    if flag_frac > 0.0:
        rng = np.random.default_rng(seed + 77)
        valid = torch.from_numpy(gap_flags(n_t, flag_frac, flag_mean_len, rng)).to(device)
    meta = dict(f_knee=f_knee, alpha=alpha, sigma=sigma, sky_sigma=dict(sky_sigma),
                flag_frac=flag_frac, seed=seed, first_sample=first_sample,
                f_samp=scan.f_samp)
    return Problem(n_t, nside, kinds, baseline_len, pix, c32, s32, y, sky, valid, c64, s64, meta)


# --------------------------------------------------------------------------------------
# Workloads.  Sizes, scan, sky and noise shapes follow the paper's B-Machine and LATTE
# setups (Sects. 2, 5, 7 and Conclusion), scaled to the 50 Hz synthetic scan.

CONFIGS = {
    # 2^20 samples, q+u outputs, nside 64, 10 s baselines
    1: dict(n_t=1 << 20, nside=64, kinds=("q", "u"), baseline_len=500, f_knee=0.1,
            alpha=1.7, sky_sigma={"Q": 1.0, "U": 1.0}),
    # 30 days of one B-Machine-like channel: I, q, u outputs, nside 256, 60 s baselines
    2: dict(n_t=130_000_000, nside=256, kinds=("I", "q", "u"), baseline_len=3000,
            f_knee=0.05, alpha=1.5, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0}),
    # 12 months of a LATTE-like IQU radiometer: nside 512, 1 s baselines, 2% flagged;
    # its polarisation angle turns once per 10 minutes (a modulator), without which
    # every IQU pixel matrix of a fixed-elevation scan is singular
    4: dict(n_t=1_600_000_000, nside=512, kinds=("iqu",), baseline_len=50, f_knee=0.05,
            alpha=1.5, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0}, flag_frac=0.02,
            scan=ScanParams(pol_rotation_period=600.0)),
}

WORKLOAD_NAMES = {
    1: "qu-nside64-2^20-L500",
    2: "bmachine30d-Iqu-nside256-1.3e8-L3000",
    4: "latte12m-iqu-nside512-1.6e9-L50-flag2pct",
}


def config_problem(k: int, device="cpu", n_t: Optional[int] = None, **overrides) -> Problem:
    """Problem of workload k (seed 1000 + k); n_t may be cut to a prefix."""
    cfg = dict(CONFIGS[k])
    if n_t is not None:
        cfg["n_t"] = int(n_t)
    cfg.update(overrides)
    cfg.setdefault("seed", 1000 + k)
    return make_problem(device=device, **cfg)


def batch_configs(n_problems: int = 64, seed: int = 1003, n_min: float = 1e6,
                  n_max: float = 3e7) -> list:
    """Parameters of a batch of independent problems of uneven size.

    Lengths log-uniform in [n_min, n_max]; nside from {64, 128, 256}; baselines of
    1, 10 or 60 s (50, 500, 3000 samples); knee frequency uniform in 0.01-0.5 Hz;
    alpha 1.7; q+u outputs; each problem starts on a different day of the scan.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_problems):
        n_t = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        out.append(dict(n_t=n_t, nside=int(rng.choice([64, 128, 256])), kinds=("q", "u"),
                        baseline_len=int(rng.choice([50, 500, 3000])),
                        f_knee=float(rng.uniform(0.01, 0.5)), alpha=1.7,
                        sky_sigma={"Q": 1.0, "U": 1.0}, seed=seed * 1000 + i,
                        first_sample=int(rng.integers(0, 365)) * 86400 * 50))
    return out
