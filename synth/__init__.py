"""Seeded synthetic inputs for the destriper: scan pointing, HEALPix RING pixels,
Gaussian skies, 1/f noise and flags.

This package is the one module that both the CPU oracle and the GPU path take
inputs from.  It holds no destriping arithmetic (no binning, pixel solve, rescan
or baseline sums).
"""
from .healpix import ang2pix_ring, npix_of, pix2ang_ring, pixels_in_ring, ring_of_pix
from .noise import gap_flags, one_over_f
from .problems import (CONFIGS, KIND_CODE, KINDS, WORKLOAD_NAMES, Problem, batch_configs,
                       components, config_problem, make_problem, n_baselines)
from .scan import ScanParams, scan_pointing

__all__ = [
    "ang2pix_ring", "npix_of", "pix2ang_ring", "pixels_in_ring", "ring_of_pix",
    "gap_flags", "one_over_f", "CONFIGS", "KIND_CODE", "KINDS", "WORKLOAD_NAMES",
    "Problem", "batch_configs", "components", "config_problem", "make_problem",
    "n_baselines", "ScanParams", "scan_pointing",
]
