"""Float64 CPU oracle of the paper's time-domain steps around the destriper.

TEST INFRASTRUCTURE ONLY (like core.py): imported by the test suite and the
benchmark's CPU legs, never by the product path, and sharing no code with the
CUDA library.

  * White-noise gap filling (Sect. 2, data description): every flagged sample
    of an output is replaced by Gaussian white noise with the mean and standard
    deviation of that output's good samples in the same day of data.
  * Timeline amplitude spectra (Sect. 6, frequency domain): the amplitude
    spectrum of y and of the baseline-removed y - F~ a, averaged over frequency
    bins of linearly increasing length.

Readings of points the paper leaves open (also listed in the design notes):
  * "Day": a block of block_len consecutive samples (86400 s times the sampling
    rate in the workloads), the last block shorter.  The standard deviation is the
    population one (ddof = 0).  A block without good samples fills its flagged
    samples with 0.
  * The random draws: one counter-based generator, Philox4x32-10 (Salmon, Moraes,
    Dror & Shaw 2011, "Parallel random numbers: as easy as 1, 2, 3"), with the
    counter (t mod 2^32, t div 2^32, o, 0) for sample t of output o and the key
    (seed mod 2^32, seed div 2^32); its first two words u0, u1 give the uniforms
    (u + 1/2) 2^-32 and one normal draw by Box-Muller,
    z = sqrt(-2 ln u0) cos(2 pi u1).
  * The spectrum: non-overlapping segments of seg_len samples (the tail that does
    not fill a segment is dropped), no window, the one-sided power spectral density
    P(f_k) = 2 |X_k|^2 / (f_samp seg_len) averaged over segments (k = seg_len / 2,
    the Nyquist term, and k = 0 are not doubled), the amplitude sqrt(P); the bins
    cover k = 1 .. seg_len / 2 with edges e_j = floor(K j (j + 1) / (n (n + 1))),
    K = seg_len / 2, bin j holding k = e_{j-1} + 1 .. e_j, so that bin j is about j
    times as long as the first; each bin reports the mean frequency and the mean
    amplitude of its k.
"""
from __future__ import annotations

import numpy as np

# Philox4x32 constants (multipliers and Weyl key increments) of the published
# generator.
_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of counters (uint32 words) and a key.

    Each round: (hi0, lo0) = M0 * c0 and (hi1, lo1) = M1 * c2 as 64-bit products;
    the new counter is (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then the key is
    bumped by the Weyl constants (not after the last round)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint32) for v in (c0, c1, c2, c3))
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    for r in range(10):
        p0 = _M0 * c0.astype(np.uint64)
        p1 = _M1 * c2.astype(np.uint64)
        hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & _MASK32).astype(np.uint32)
        hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & _MASK32).astype(np.uint32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            with np.errstate(over="ignore"):
                k0 = np.uint32(k0 + _W0)
                k1 = np.uint32(k1 + _W1)
    return c0, c1, c2, c3


def normal_draws(t, o, seed):
    """Standard normal draw for samples t (int array) of output o (see the module
    docstring for the counter, key and Box-Muller step)."""
    t = np.asarray(t, dtype=np.uint64)
    c0 = (t & _MASK32).astype(np.uint32)
    c1 = (t >> np.uint64(32)).astype(np.uint32)
    c2 = np.full(t.shape, o, dtype=np.uint32)
    c3 = np.zeros(t.shape, dtype=np.uint32)
    seed = int(seed)
    w0, w1, _, _ = philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u0 = (w0.astype(np.float64) + 0.5) * 2.0 ** -32
    u1 = (w1.astype(np.float64) + 0.5) * 2.0 ** -32
    return np.sqrt(-2.0 * np.log(u0)) * np.cos(2.0 * np.pi * u1)


def gapfill(y, valid, block_len, seed):
    """White-noise gap filling (Sect. 2): y [n_o, n_t] float64, valid [n_t] (1 good).
    Returns a copy with every flagged sample of every output replaced by
    mean + std * z over its block's good samples."""
    y = np.array(y, dtype=np.float64, copy=True).reshape(-1, np.asarray(valid).shape[0])
    n_o, n_t = y.shape
    good = np.asarray(valid).astype(bool)
    for o in range(n_o):
        for start in range(0, n_t, block_len):
            end = min(start + block_len, n_t)
            g = good[start:end]
            bad = np.nonzero(~g)[0] + start
            if bad.size == 0:
                continue
            if g.any():
                vals = y[o, start:end][g]
                mu = vals.mean()
                sd = np.sqrt(np.mean((vals - mu) ** 2))
                y[o, bad] = mu + sd * normal_draws(bad, o, seed)
            else:
                y[o, bad] = 0.0
    return y


def bin_edges(seg_len, n_bins):
    """Edges e_0 = 0 < e_1 < ... < e_n = K of the linearly growing bins."""
    K = seg_len // 2
    j = np.arange(n_bins + 1, dtype=np.int64)
    e = (K * j * (j + 1)) // (n_bins * (n_bins + 1))
    if np.any(np.diff(e) < 1):
        raise ValueError("too many bins for the segment length")
    return e


def psd(z, f_samp, seg_len):
    """One-sided power spectral density of z, averaged over its whole segments
    (k = 0 .. seg_len / 2); returns (frequencies, P)."""
    z = np.asarray(z, dtype=np.float64)
    n_seg = z.shape[0] // seg_len
    if n_seg < 1:
        raise ValueError("timeline shorter than one segment")
    X = np.fft.rfft(z[: n_seg * seg_len].reshape(n_seg, seg_len), axis=1)
    P = np.mean(np.abs(X) ** 2, axis=0) * 2.0 / (f_samp * seg_len)
    P[0] /= 2.0
    if seg_len % 2 == 0:
        P[-1] /= 2.0
    return np.arange(P.shape[0]) * f_samp / seg_len, P


def amplitude_spectrum(z, f_samp, seg_len, n_bins):
    """Binned amplitude spectral density of one timeline z (Sect. 6 reading above).
    Returns (frequencies [n_bins], amplitudes [n_bins])."""
    freq, P = psd(z, f_samp, seg_len)
    amp = np.sqrt(P)
    e = bin_edges(seg_len, n_bins)
    fb = np.array([freq[e[j] + 1: e[j + 1] + 1].mean() for j in range(n_bins)])
    ab = np.array([amp[e[j] + 1: e[j + 1] + 1].mean() for j in range(n_bins)])
    return fb, ab


def destriped_timeline(y, a, baseline_len):
    """y - F~ a: each output's timeline minus its baselines (Sect. 6, frequency
    domain: the baseline-removed signal)."""
    y = np.asarray(y, dtype=np.float64)
    y = y.reshape(-1, y.shape[-1])
    n_t = y.shape[1]
    a = np.asarray(a, dtype=np.float64).reshape(y.shape[0], -1)
    return y - a[:, np.arange(n_t) // baseline_len]
