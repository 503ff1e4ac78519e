"""HEALPix RING pixelisation, written from the published construction of the grid
(Gorski et al. 2005, ApJ 622, 759: Sect. 4 and the RING-scheme pixel index).

The sky is split into 12 base quadrilaterals of equal area, each subdivided into
nside x nside pixels.  Pixel centres sit on 4*nside - 1 rings of constant
colatitude.  In the polar caps (|z| > 2/3, z = cos(theta)) ring i (counted from the
nearest pole) holds 4*i pixels; in the equatorial belt every ring holds 4*nside
pixels and alternate rings are shifted by half a pixel.  RING indices run ring by
ring from the north pole, east-ward in longitude within a ring.

The maps of the destriping paper are HEALPix maps (paper Sect. 3, Eq. destmodel);
the build only needs pixel indices as *inputs* (the pointing matrix P), so this
module belongs to the synthetic input generator, not to the method.

All functions take and return torch tensors, and work on any device.
"""
from __future__ import annotations

import math

import torch


def npix_of(nside: int) -> int:
    """Number of pixels of a HEALPix map: 12 base pixels of nside^2 each."""
    return 12 * nside * nside


def check_nside(nside: int) -> None:
    if nside < 1 or (nside & (nside - 1)) != 0 or nside > (1 << 13):
        raise ValueError(f"nside must be a power of two in [1, 8192], got {nside}")


def ang2pix_ring(nside: int, theta: torch.Tensor, phi: torch.Tensor) -> torch.Tensor:
    """RING pixel index (int64) of the pixel containing (theta, phi), in radians.

    theta is the colatitude in [0, pi], phi the longitude (any value; it is wrapped
    to [0, 2 pi)).  Computation is in float64.
    """
    check_nside(nside)
    theta = theta.to(torch.float64)
    phi = torch.remainder(phi.to(torch.float64), 2.0 * math.pi)
    z = torch.cos(theta)
    za = z.abs()
    # longitude in units of a quarter turn, in [0, 4)
    tt = phi * (2.0 / math.pi)
    tt = torch.where(tt >= 4.0, tt - 4.0, tt)
    ns = float(nside)
    npix = npix_of(nside)
    ncap = 2 * nside * (nside - 1)  # pixels in the north polar cap

    # --- equatorial belt: pixel edges are the lines phi/(pi/2) +- 3/4 z * ... ----
    t1 = ns * (0.5 + tt)
    t2 = ns * z * 0.75
    jp = torch.floor(t1 - t2).to(torch.int64)  # index of the ascending edge line
    jm = torch.floor(t1 + t2).to(torch.int64)  # index of the descending edge line
    ir_eq = nside + 1 + jp - jm  # ring number counted from z = 2/3, in [1, 2 nside + 1]
    kshift = 1 - (ir_eq & 1)  # rings with even ir_eq are shifted by half a pixel
    ip_eq = torch.div(jp + jm - nside + kshift + 1, 2, rounding_mode="floor")
    ip_eq = torch.remainder(ip_eq, 4 * nside)
    pix_eq = ncap + (ir_eq - 1) * (4 * nside) + ip_eq

    # --- polar caps: rings of 4*i pixels, i from the nearest pole -----------------
    tp = tt - torch.floor(tt)
    tmp = ns * torch.sqrt(torch.clamp(3.0 * (1.0 - za), min=0.0))
    jp_c = torch.floor(tp * tmp).to(torch.int64)
    jm_c = torch.floor((1.0 - tp) * tmp).to(torch.int64)
    ir_c = jp_c + jm_c + 1  # ring number from the nearest pole, in [1, nside]
    ip_c = torch.floor(tt * ir_c.to(torch.float64)).to(torch.int64)
    ip_c = torch.remainder(ip_c, 4 * ir_c)
    pix_n = 2 * ir_c * (ir_c - 1) + ip_c
    pix_s = npix - 2 * ir_c * (ir_c + 1) + ip_c
    pix_cap = torch.where(z > 0, pix_n, pix_s)

    return torch.where(za <= 2.0 / 3.0, pix_eq, pix_cap)


def _cap_ring(q: torch.Tensor) -> torch.Tensor:
    """Ring number i >= 1 (from the nearest pole) with 2 i (i - 1) < q <= 2 i (i + 1).

    In a polar cap ring i holds 4 i pixels, so the first i rings hold 2 i (i + 1)
    pixels; q is the 1-based rank of a pixel counted from that pole.
    """
    i = torch.floor((1.0 + torch.sqrt(torch.clamp(2.0 * q.to(torch.float64) - 1.0, min=1.0))) / 2.0)
    i = i.to(torch.int64)
    i = torch.where(2 * i * (i - 1) >= q, i - 1, i)
    i = torch.where(2 * i * (i + 1) < q, i + 1, i)
    return torch.clamp(i, min=1)


def ring_of_pix(nside: int, pix: torch.Tensor):
    """(ring index i in [1, 4 nside - 1] from the north pole, position j in [1, n_i])."""
    check_nside(nside)
    pix = pix.to(torch.int64)
    npix = npix_of(nside)
    ncap = 2 * nside * (nside - 1)
    # north cap, 1-based rank from the north pole
    i_n = _cap_ring(pix + 1)
    j_n = pix - 2 * i_n * (i_n - 1) + 1
    # equatorial belt (rings nside .. 3 nside, 4 nside pixels each)
    ip = pix - ncap
    i_e = torch.div(ip, 4 * nside, rounding_mode="floor") + nside
    j_e = torch.remainder(ip, 4 * nside) + 1
    # south cap, 1-based rank from the south pole; positions still run east-ward
    ps = npix - pix
    i_s = _cap_ring(ps)
    j_s = 2 * i_s * (i_s + 1) + 1 - ps
    ring = torch.where(pix < ncap, i_n, torch.where(pix < npix - ncap, i_e, 4 * nside - i_s))
    pos = torch.where(pix < ncap, j_n, torch.where(pix < npix - ncap, j_e, j_s))
    return ring, pos


def pix2ang_ring(nside: int, pix: torch.Tensor):
    """Centre (theta, phi) of RING pixels, from the ring/position construction."""
    ring, pos = ring_of_pix(nside, pix)
    ns = float(nside)
    i = ring.to(torch.float64)
    j = pos.to(torch.float64)
    # north cap: z = 1 - i^2 / (3 nside^2), phi = pi / (2 i) * (j - 1/2)
    z_n = 1.0 - i * i / (3.0 * ns * ns)
    phi_n = math.pi / (2.0 * i) * (j - 0.5)
    # equatorial belt: z = 4/3 - 2 i / (3 nside).  Rings with (i - nside) even
    # continue the cap pattern (first centre half a pixel east of phi = 0); the
    # others are shifted by half a pixel, so their first centre sits on phi = 0.
    s = torch.remainder(ring - nside + 1, 2).to(torch.float64)
    z_e = 4.0 / 3.0 - 2.0 * i / (3.0 * ns)
    phi_e = math.pi / (2.0 * ns) * (j - 1.0 + s / 2.0)
    # south cap mirrors the north cap with i' = 4 nside - i
    i_s = 4.0 * ns - i
    z_s = -(1.0 - i_s * i_s / (3.0 * ns * ns))
    phi_s = math.pi / (2.0 * i_s) * (j - 0.5)
    north = ring < nside
    south = ring > 3 * nside
    z = torch.where(north, z_n, torch.where(south, z_s, z_e))
    phi = torch.where(north, phi_n, torch.where(south, phi_s, phi_e))
    return torch.arccos(torch.clamp(z, -1.0, 1.0)), phi


def pixels_in_ring(nside: int, ring: int) -> int:
    """Number of pixels in ring `ring` (1-based from the north pole)."""
    if ring < nside:
        return 4 * ring
    if ring <= 3 * nside:
        return 4 * nside
    return 4 * (4 * nside - ring)
