"""Float64 CPU oracle of the destriping method.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline / reference arm, never by the product path.  It shares
no code with the CUDA library.  See core.py for the method and its readings.
"""
from .core import (OraclePlan, apply_A, apply_Z, baseline_has_data, baseline_sums,
                       bin_map, cg, components, destripe, expand, gauge, hitmap, make_plan,
                       pixel_cut, pixel_matrices, pixel_solve, pixel_sums, rescan, rhs,
                       row_coefficients)

__all__ = [
    "OraclePlan", "apply_A", "apply_Z", "baseline_has_data", "baseline_sums", "bin_map",
    "cg", "components", "destripe", "expand", "gauge", "hitmap", "make_plan", "pixel_cut",
    "pixel_matrices", "pixel_solve", "pixel_sums", "rescan", "rhs", "row_coefficients",
]
