"""Ground-based spin scan: fixed elevation, constant azimuth rate, Earth rotation.

The paper's instrument spins about its vertical axis at fixed 45 deg elevation and
gets its crossing points from the rotation of the sky (paper Sect. 5, scanning
strategy).  This module turns sample times into equatorial pointing (colatitude,
right ascension) and the parallactic angle psi that orients the polarimeter
(paper Sect. 3, footnote on the parallactic angle), with textbook spherical
astronomy:

    sin(dec) = sin(el) sin(lat) + cos(el) cos(lat) cos(az)
    H        = atan2(-sin(az) cos(el), sin(el) cos(lat) - cos(el) sin(lat) cos(az))
    RA       = LST - H
    psi      = atan2(sin(H), tan(lat) cos(dec) - sin(dec) cos(H))

Azimuth is measured from north through east; H is the hour angle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch


@dataclass(frozen=True)
class ScanParams:
    f_samp: float = 50.0  # Hz
    spin_period: float = 60.0  # s per azimuth revolution
    elevation_deg: float = 45.0
    latitude_deg: float = 34.4
    az0: float = 0.0  # rad, azimuth at t = 0 (north)
    lst0: float = 0.0  # rad, local sidereal time at t = 0
    sidereal_day: float = 86164.0905  # s
    # Period (s) of a continuously rotating polarisation angle added to the
    # parallactic angle (a polarisation modulator); 0 = none.  A single detector
    # at fixed elevation sees each pixel at only two parallactic angles (rising
    # and setting), which leaves the 3x3 I/Q/U pixel matrix rank 2.
    pol_rotation_period: float = 0.0


def scan_pointing(n: int, params: ScanParams = ScanParams(), first_sample: int = 0,
                  device="cpu"):
    """Pointing of samples first_sample .. first_sample + n - 1.

    Returns (theta, phi, psi) float64 tensors: colatitude, right ascension (both
    rad, HEALPix convention) and parallactic angle (rad).
    """
    k = torch.arange(first_sample, first_sample + n, dtype=torch.float64, device=device)
    t = k / params.f_samp
    az = params.az0 + (2.0 * math.pi / params.spin_period) * t
    lst = params.lst0 + (2.0 * math.pi / params.sidereal_day) * t
    el = math.radians(params.elevation_deg)
    lat = math.radians(params.latitude_deg)
    sin_el, cos_el = math.sin(el), math.cos(el)
    sin_lat, cos_lat = math.sin(lat), math.cos(lat)
    cos_az = torch.cos(az)
    sin_az = torch.sin(az)
    sin_dec = torch.clamp(sin_el * sin_lat + cos_el * cos_lat * cos_az, -1.0, 1.0)
    dec = torch.arcsin(sin_dec)
    ha = torch.atan2(-sin_az * cos_el, sin_el * cos_lat - cos_el * sin_lat * cos_az)
    ra = torch.remainder(lst - ha, 2.0 * math.pi)
    psi = torch.atan2(torch.sin(ha), math.tan(lat) * torch.cos(dec) - sin_dec * torch.cos(ha))
    if params.pol_rotation_period > 0.0:
        psi = psi + (2.0 * math.pi / params.pol_rotation_period) * t
    theta = 0.5 * math.pi - dec
    return theta, ra, psi
