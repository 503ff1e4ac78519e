"""Pins of the synthetic input generator: HEALPix RING geometry (Gorski et al.
2005), the spin-scan spherical astronomy, the 1/f spectrum (paper Eq. 1fnoise) and
the flag recipe."""
import math

import numpy as np
import pytest
import torch

from synth import (ScanParams, ang2pix_ring, gap_flags, make_problem, npix_of, one_over_f,
                   pix2ang_ring, pixels_in_ring, ring_of_pix, scan_pointing)


@pytest.mark.parametrize("nside", [1, 2, 4, 64, 512])
def test_npix_and_range(nside):
    assert npix_of(nside) == 12 * nside * nside
    g = torch.Generator().manual_seed(nside)
    z = torch.rand(20000, generator=g, dtype=torch.float64) * 2 - 1
    phi = torch.rand(20000, generator=g, dtype=torch.float64) * 8 * math.pi - 4 * math.pi
    p = ang2pix_ring(nside, torch.arccos(z), phi)
    assert int(p.min()) >= 0 and int(p.max()) < npix_of(nside)


def test_base_pixel_centres():
    # The 12 base pixels: 4 around z = 2/3 at phi = 45, 135, 225, 315 deg, 4 on the
    # equator at phi = 0, 90, 180, 270 deg, 4 around z = -2/3 (Gorski et al. 2005).
    th, ph = pix2ang_ring(1, torch.arange(12))
    z = torch.cos(th)
    exp_z = [2 / 3] * 4 + [0.0] * 4 + [-2 / 3] * 4
    exp_phi = [45, 135, 225, 315, 0, 90, 180, 270, 45, 135, 225, 315]
    assert np.allclose(z.numpy(), exp_z, atol=1e-12)
    assert np.allclose(np.degrees(ph.numpy()), exp_phi, atol=1e-9)
    assert (ang2pix_ring(1, th, ph) == torch.arange(12)).all()


@pytest.mark.parametrize("nside", [1, 2, 8, 32])
def test_rings_are_contiguous_with_published_counts(nside):
    pix = torch.arange(npix_of(nside))
    ring, pos = ring_of_pix(nside, pix)
    counts = torch.bincount(ring, minlength=4 * nside)[1:]
    exp = [pixels_in_ring(nside, i) for i in range(1, 4 * nside)]
    assert counts.tolist() == exp
    assert sum(exp) == npix_of(nside)
    # RING order: ring index never decreases, positions count 1..n_i within a ring
    assert (ring[1:] >= ring[:-1]).all()
    first = torch.ones_like(pos, dtype=torch.bool)
    first[1:] = ring[1:] != ring[:-1]
    assert (pos[first] == 1).all()
    assert (pos[~first] == pos[torch.nonzero(~first).squeeze(1) - 1] + 1).all()
    # every pixel of a ring has the same colatitude
    th, _ = pix2ang_ring(nside, pix)
    for i in range(1, 4 * nside):
        zi = torch.cos(th[ring == i])
        assert float(zi.max() - zi.min()) < 1e-12


@pytest.mark.parametrize("nside", [1, 4, 64, 512])
def test_centre_round_trip(nside):
    pix = torch.arange(npix_of(nside))
    th, ph = pix2ang_ring(nside, pix)
    assert (ang2pix_ring(nside, th, ph) == pix).all()


@pytest.mark.parametrize("nside", [1, 4, 16])
def test_equal_area(nside):
    # uniform points on the sphere fill every pixel equally (chi^2 within 5 sigma)
    g = torch.Generator().manual_seed(7)
    n = 1_000_000
    z = torch.rand(n, generator=g, dtype=torch.float64) * 2 - 1
    phi = torch.rand(n, generator=g, dtype=torch.float64) * 2 * math.pi
    c = torch.bincount(ang2pix_ring(nside, torch.arccos(z), phi), minlength=npix_of(nside)).double()
    e = n / npix_of(nside)
    chi2 = float(((c - e) ** 2 / e).sum())
    dof = npix_of(nside) - 1
    assert abs(chi2 - dof) < 5 * math.sqrt(2 * dof) + 5


def test_scan_closed_forms():
    sp = ScanParams()
    lat, el = math.radians(sp.latitude_deg), math.radians(sp.elevation_deg)
    # az = 0 (north): dec = lat + el, hour angle 0 so RA = LST = 0
    th, ra, psi = scan_pointing(1, sp, 0)
    assert abs((math.pi / 2 - float(th[0])) - (lat + el)) < 1e-12
    assert min(abs(float(ra[0])), abs(float(ra[0]) - 2 * math.pi)) < 1e-12
    # half a spin later (az = 180 deg, south): dec = lat - el
    half = int(sp.spin_period * sp.f_samp / 2)
    th, ra, psi = scan_pointing(1, sp, half)
    assert abs((math.pi / 2 - float(th[0])) - (lat - el)) < 1e-9
    # a day of scanning stays inside the declination band [lat - el, lat + el]
    th, ra, psi = scan_pointing(86400 * 5, ScanParams(f_samp=5.0), 0)
    dec = math.pi / 2 - th
    assert float(dec.min()) >= lat - el - 1e-9 and float(dec.max()) <= lat + el + 1e-9
    assert float(psi.abs().max()) <= math.pi + 1e-12


def test_one_over_f_spectrum():
    n, fs, fk, alpha, sigma = 1 << 18, 50.0, 0.5, 1.5, 1.0
    spec = torch.zeros(n // 2 + 1, dtype=torch.float64)
    for seed in range(8):
        g = torch.Generator().manual_seed(seed)
        x = one_over_f(n, fs, fk, alpha, sigma, g)
        assert abs(float(x.mean())) < 1e-12  # zero-frequency bin removed
        spec += torch.fft.rfft(x).abs() ** 2 / n
    spec /= 8
    f = torch.fft.rfftfreq(n, 1 / fs)
    model = sigma ** 2 * (1 + (fk / f[1:]) ** alpha)
    ratio = spec[1:] / model
    hi = (f[1:] > 5.0)
    lo = (f[1:] > 0.02) & (f[1:] < 0.1)
    assert abs(float(ratio[hi].mean()) - 1) < 0.02
    assert abs(float(ratio[lo].mean()) - 1) < 0.15


def test_gap_flags_exact_fraction():
    rng = np.random.default_rng(3)
    v = gap_flags(1_000_000, 0.02, 500, rng)
    assert int((v == 0).sum()) == 20000
    starts = np.flatnonzero(np.diff(np.concatenate([[1], v.astype(np.int64)])) == -1)
    assert 20 < len(starts) < 100  # geometric gaps of mean 500


def test_problem_signal_is_in_model_range():
    # the signal part of y uses the stored float32 trig exactly
    p = make_problem(5000, 16, ("q", "u", "I"), 50, noise=False, seed=5)
    q = p.sky[1, p.pix.long()] * p.c32.double() + p.sky[2, p.pix.long()] * p.s32.double()
    assert torch.equal(p.y[0], q)
    assert torch.equal(p.y[2], p.sky[0, p.pix.long()])
