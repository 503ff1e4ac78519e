"""Noise and flag synthesis for the synthetic timelines.

1/f noise follows the spectrum of the paper's Eq. 1fnoise,
P(f) ~ sigma^2 [1 + (f_k / f)^alpha]: seeded white noise of standard deviation
sigma is Fourier transformed, each positive-frequency bin is scaled by
sqrt(1 + (f_k / f)^alpha), the zero-frequency bin is set to 0 and the result is
transformed back.  Long timelines are built from independent segments.

Flags stand in for the bad-data flags of the paper's timelines (Sect. 2): a set
fraction of samples is marked invalid in contiguous gaps of geometric length.
"""
from __future__ import annotations

import numpy as np
import torch

SEGMENT = 1 << 27  # samples per independent FFT segment for long timelines


def one_over_f(n: int, f_samp: float, f_knee: float, alpha: float, sigma: float,
               gen: torch.Generator, device="cpu") -> torch.Tensor:
    """float64 1/f + white noise timeline of length n."""
    out = torch.empty(n, dtype=torch.float64, device=device)
    pos = 0
    seg = n if n <= (1 << 28) else SEGMENT
    while pos < n:
        m = min(seg, n - pos)
        w = torch.randn(m, generator=gen, dtype=torch.float64, device=device) * sigma
        if f_knee > 0.0 and m > 1:
            spec = torch.fft.rfft(w)
            f = torch.fft.rfftfreq(m, d=1.0 / f_samp, dtype=torch.float64, device=device)
            scale = torch.ones_like(f)
            scale[1:] = torch.sqrt(1.0 + (f_knee / f[1:]) ** alpha)
            scale[0] = 0.0
            spec = spec * scale
            w = torch.fft.irfft(spec, n=m)
            del spec
        out[pos:pos + m] = w
        pos += m
    return out


def gap_flags(n: int, frac: float, mean_len: float, rng: np.random.Generator) -> np.ndarray:
    """uint8 valid flags (1 = good) with round(frac * n) samples flagged.

    Gap lengths are geometric with the given mean; the last one is cut so that the
    flagged count is exact.  Gaps are placed without overlap by splitting the good
    samples into (n_gaps + 1) runs at uniform random cut points.
    """
    valid = np.ones(n, dtype=np.uint8)
    target = int(round(frac * n))
    if target <= 0:
        return valid
    lens = []
    total = 0
    p = 1.0 / max(mean_len, 1.0)
    while total < target:
        g = int(rng.geometric(p))
        g = min(g, target - total)
        lens.append(g)
        total += g
    n_good = n - target
    cuts = np.sort(rng.integers(0, n_good + 1, size=len(lens)))
    good_runs = np.diff(np.concatenate([[0], cuts, [n_good]]))
    pos = 0
    for i, g in enumerate(lens):
        pos += int(good_runs[i])
        valid[pos:pos + g] = 0
        pos += g
    return valid
