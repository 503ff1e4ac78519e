"""Device pointing of an analytic scan (destripe_scan_pointing) against the
seeded input generator that every other test and the benchmark use
(synth.scan + synth.healpix, evaluated by torch on the same GPU): pixels
bit-exact, cos 2psi / sin 2psi bit-exact, over a whole 30-day B-Machine-like
scan at nside 256 and the LATTE-like scan with its modulator at nside 512, from
several starting samples."""
import pytest
import torch

import paper_1309_5609_gb300 as ds
from synth import ScanParams
from synth.healpix import ang2pix_ring
from synth.scan import scan_pointing

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def reference(n, scan, first, nside):
    theta, phi, psi = scan_pointing(n, scan, first, device=DEV)
    pix = ang2pix_ring(nside, theta, phi).to(torch.int32)
    return pix, torch.cos(2.0 * psi).to(torch.float32), torch.sin(2.0 * psi).to(torch.float32)


@pytest.mark.parametrize("scan,nside,n_total", [
    (ScanParams(), 256, 130_000_000),
    (ScanParams(pol_rotation_period=600.0), 512, 40_000_000),
    (ScanParams(f_samp=5.0, sidereal_day=7200.0), 8, 3_000_000),
], ids=["bmachine30d_nside256", "latte_modulated_nside512", "fast_sky_nside8"])
def test_scan_pointing_matches_the_generator(scan, nside, n_total):
    chunk = 1 << 24
    mism = [0, 0, 0]
    for first in range(0, n_total, chunk):
        n = min(chunk, n_total - first)
        pr, cr, sr = reference(n, scan, first, nside)
        p, c, s = ds.destripe_scan_pointing(scan, first, n, nside)
        mism[0] += int((p != pr).sum())
        mism[1] += int((c != cr).sum())
        mism[2] += int((s != sr).sum())
    assert mism == [0, 0, 0], mism


def test_scan_pointing_rejects_bad_scans():
    with pytest.raises(ds.DestripeError):
        ds.destripe_scan_pointing(ScanParams(f_samp=0.0), 0, 10, 64)
    with pytest.raises(ds.DestripeError):
        ds.destripe_scan_pointing(ScanParams(), 0, 10, 63)
