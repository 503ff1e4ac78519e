"""Pins of the oracle's gap filling and timeline spectra (oracle/diagnostics.py)
against what the publications and the mathematics fix:

  * Philox4x32-10 against its published known-answer vectors (tests/golden);
  * the normal draws: Box-Muller of the generator's words, standard normal by a
    Kolmogorov-Smirnov test and by their moments;
  * gap filling (paper Sect. 2): good samples untouched; a flagged sample in a day
    whose good samples are 1 and 3 becomes exactly 2 + 1 * z (population standard
    deviation); each day uses its own statistics; a day without good samples is
    filled with 0; the fill is reproducible from the seed and differs per output;
  * the spectrum (paper Sect. 6): Parseval (the one-sided density integrates to
    the mean square), a cosine on a Fourier frequency puts A^2 N / (2 f_samp) in its
    bin, white noise of variance s^2 has the flat density 2 s^2 / f_samp, and the
    bins partition 1 .. N/2 with lengths growing linearly.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import diagnostics as dg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")


def test_philox_known_answers():
    kat = json.load(open(GOLDEN))
    for v in kat["vectors"]:
        c = [np.array([int(x, 16)], dtype=np.uint32) for x in v["counter"]]
        k = [int(x, 16) for x in v["key"]]
        out = dg.philox4x32_10(*c, *k)
        assert [f"{int(w[0]):08x}" for w in out] == v["out"]


def test_normal_draws_are_standard_normal():
    scipy_stats = pytest.importorskip("scipy.stats")
    t = np.arange(200_000)
    z = dg.normal_draws(t, 1, seed=12345)
    assert abs(z.mean()) < 5 / math.sqrt(t.size)
    assert abs(z.std() - 1.0) < 5 / math.sqrt(2 * t.size)
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-3
    # one Box-Muller step of the generator's first two words
    w = dg.philox4x32_10(np.uint32([7]), np.uint32([0]), np.uint32([1]), np.uint32([0]),
                         12345, 0)
    u0, u1 = (float(w[0][0]) + 0.5) / 2 ** 32, (float(w[1][0]) + 0.5) / 2 ** 32
    assert dg.normal_draws(np.array([7]), 1, 12345)[0] == pytest.approx(
        math.sqrt(-2 * math.log(u0)) * math.cos(2 * math.pi * u1), rel=1e-15)
    # outputs and seeds draw different numbers
    assert not np.allclose(dg.normal_draws(t[:100], 0, 1), dg.normal_draws(t[:100], 1, 1))
    assert not np.allclose(dg.normal_draws(t[:100], 0, 1), dg.normal_draws(t[:100], 0, 2))


def test_gapfill_uses_each_days_good_samples():
    n_t, day = 30, 10
    y = np.zeros((2, n_t))
    valid = np.ones(n_t, dtype=np.uint8)
    # day 0: good samples 1 and 3 (mean 2, population std 1), the rest flagged
    y[:, 0], y[:, 1] = 1.0, 3.0
    valid[2:10] = 0
    # day 1: all good; day 2: no good sample
    y[:, 10:20] = 100.0 + np.arange(10)
    valid[20:30] = 0
    y[:, 20:30] = np.nan
    out = dg.gapfill(y, valid, day, seed=99)
    flagged = np.arange(2, 10)
    for o in range(2):
        assert np.array_equal(out[o, :2], y[o, :2])
        assert np.allclose(out[o, flagged], 2.0 + 1.0 * dg.normal_draws(flagged, o, 99),
                           rtol=0, atol=1e-15)
        assert np.array_equal(out[o, 10:20], y[o, 10:20])
        assert np.array_equal(out[o, 20:30], np.zeros(10))
    assert np.array_equal(dg.gapfill(y, valid, day, seed=99), out)
    assert not np.allclose(out[0, flagged], out[1, flagged])


def test_gapfill_statistics_follow_the_good_samples():
    rng = np.random.default_rng(0)
    n_t, day = 400_000, 200_000
    y = np.concatenate([rng.normal(5.0, 2.0, day), rng.normal(-3.0, 0.5, day)])[None, :]
    valid = (rng.random(n_t) > 0.3).astype(np.uint8)
    out = dg.gapfill(y, valid, day, seed=3)
    for d, (mu, sd) in enumerate([(5.0, 2.0), (-3.0, 0.5)]):
        sl = slice(d * day, (d + 1) * day)
        filled = out[0, sl][valid[sl] == 0]
        assert abs(filled.mean() - mu) < 6 * sd / math.sqrt(filled.size)
        assert abs(filled.std() - sd) < 6 * sd / math.sqrt(2 * filled.size)


def test_psd_parseval_and_white_level():
    rng = np.random.default_rng(1)
    fs, N = 50.0, 4096
    z = rng.normal(0.0, 1.7, 40 * N)
    f, P = dg.psd(z, fs, N)
    # Parseval per segment, averaged: sum_k P_k df = mean of z^2
    seg = z.reshape(40, N)
    assert np.sum(P) * fs / N == pytest.approx(np.mean(seg ** 2), rel=1e-12)
    # flat density 2 s^2 / fs away from the ends
    assert np.mean(P[1:-1]) == pytest.approx(2 * 1.7 ** 2 / fs, rel=0.02)
    assert f[1] == pytest.approx(fs / N) and f[-1] == pytest.approx(fs / 2)


def test_psd_of_a_cosine_on_a_fourier_frequency():
    fs, N, k0, A = 20.0, 1024, 37, 3.0
    t = np.arange(4 * N)
    z = A * np.cos(2 * np.pi * k0 * t / N)
    f, P = dg.psd(z, fs, N)
    assert P[k0] == pytest.approx(A ** 2 * N / (2 * fs), rel=1e-12)
    assert np.max(np.delete(P, k0)) < 1e-20 * P[k0]


def test_bins_grow_linearly_and_cover_the_spectrum():
    for N, n in [(4096, 20), (1 << 16, 60), (1000, 10)]:
        e = dg.bin_edges(N, n)
        assert e[0] == 0 and e[-1] == N // 2
        lens = np.diff(e)
        assert np.all(lens >= 1)
        j = np.arange(1, n + 1)
        assert np.allclose(lens, (N // 2) * 2 * j / (n * (n + 1)), atol=1.0)
    f, a = dg.amplitude_spectrum(np.random.default_rng(2).normal(0, 1, 8 * 4096), 50.0, 4096, 20)
    assert np.all(np.diff(f) > 0)
    assert np.allclose(a, math.sqrt(2 / 50.0), rtol=0.15)


def test_destriped_timeline_subtracts_each_baseline():
    y = np.arange(14, dtype=np.float64).reshape(2, 7)
    a = np.array([[1.0, 2.0, 3.0], [10.0, 20.0, 30.0]])
    out = dg.destriped_timeline(y, a, 3)
    assert np.array_equal(out[0], y[0] - np.array([1, 1, 1, 2, 2, 2, 3.0]))
    assert np.array_equal(out[1], y[1] - np.array([10, 10, 10, 20, 20, 20, 30.0]))
