"""Plain float64 CPU oracle of maximum-likelihood destriping (Zonca et al. 2013).

TEST INFRASTRUCTURE ONLY.  This module is the reference the GPU kernels are checked
against.  Only the test suite, the smoke check and the benchmark's CPU-baseline /
reference arm may import it; the product path (the CUDA library and its Python
binding) never does, and it shares no code with them.

It follows the paper's statement of the method step by step, in float64, with no
blocking, fusion or reordering beyond what the equations state.  Sums over time
samples run in sample order (numpy.bincount), sums over baselines too.

Notation (paper Sect. 3):
  n_t samples, output o of a given kind, pointing p(t) (the pointing matrix P has
  one 1 per row), rows w_o(t) (the rotation matrices R), baselines a of L samples
  each (the matrix F), valid flags v(t) in {0, 1}.

Readings of points where the paper is silent or garbled (each also listed in the
design notes):
  * B = h^-1 P~^T R in Sect. 3 is read as M^-1 A_p^T V: the per-pixel weight is the
    general normal matrix M_p = sum_t v w w^T, which equals h_p I for a q+u
    polarimeter (Sect. 3, QU vs IQU weighting) and is 3x3 for IQU radiometers; the
    transpose of R is what Eqs. mapQ/mapU apply.
  * A pixel is kept when h_p > 0 and rcond(M_p) = lambda_min / lambda_max >= rcond_min;
    samples falling on a cut pixel get v = 0 everywhere (bin, rescan, baseline sums).
  * Hits count valid samples before the cut; the cut is reported as the mask.
  * The last baseline holds the n_t mod L left-over samples (n_b = ceil(n_t / L)).
  * CG (named in Sect. 3 as an alternative to GMRES) from x0 = 0, stopped on the
    recursive residual ||r_k|| / ||b|| < tol.
  * Outputs carrying I have a null mode (a common offset on all their baselines is
    absorbed by the I map).  The solution is gauge-fixed by removing the mean over
    baselines with at least one valid sample; baselines with no valid sample are 0.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

KINDS = ("I", "q", "u", "iqu")


def components(kinds) -> tuple:
    """Map components: I only, (Q, U), or (I, Q, U) when both are present."""
    has_i = any(k in ("I", "iqu") for k in kinds)
    has_p = any(k in ("q", "u", "iqu") for k in kinds)
    if has_i and has_p:
        return ("I", "Q", "U")
    if has_p:
        return ("Q", "U")
    if has_i:
        return ("I",)
    raise ValueError("no outputs")


def row_coefficients(kind: str, comps: tuple, c: np.ndarray, s: np.ndarray) -> dict:
    """Row w_o(t) of one output as {component index: coefficient array or scalar}.

    Sect. 3, rotation matrices: a q channel sees Q cos 2psi + U sin 2psi, a u
    channel -Q sin 2psi + U cos 2psi.  The I output of a polarimeter sees I alone
    (Sect. 2 and the start of Sect. 3: I is decoupled from q and u).  An IQU
    radiometer sees I + Q cos 2psi + U sin 2psi (the IQU case of Sect. 3).
    """
    ci = {k: i for i, k in enumerate(comps)}
    if kind == "I":
        return {ci["I"]: 1.0}
    if kind == "q":
        return {ci["Q"]: c, ci["U"]: s}
    if kind == "u":
        return {ci["Q"]: -s, ci["U"]: c}
    if kind == "iqu":
        return {ci["I"]: 1.0, ci["Q"]: c, ci["U"]: s}
    raise ValueError(kind)


def _as_array(coef, n):
    return np.full(n, coef, dtype=np.float64) if np.isscalar(coef) else coef


@dataclass
class OraclePlan:
    n_t: int
    npix: int
    kinds: tuple
    comps: tuple
    L: int
    n_b: int
    pix: np.ndarray  # int64 [n_t]
    c: np.ndarray  # float64 [n_t]
    s: np.ndarray  # float64 [n_t]
    valid: np.ndarray  # float64 [n_t], input flags (1 good)
    hits: np.ndarray  # int64 [npix]
    M: np.ndarray  # float64 [npix, n_c, n_c]
    rcond: np.ndarray  # float64 [npix]
    mask: np.ndarray  # bool [npix], good pixels
    Minv: np.ndarray  # float64 [npix, n_c, n_c], 0 on cut pixels
    v: np.ndarray  # float64 [n_t], effective weight after the cut

    @property
    def n_o(self):
        return len(self.kinds)

    @property
    def n_c(self):
        return len(self.comps)


def hitmap(pix, valid, npix):
    """h = P^T P (Sect. 3): number of valid samples per pixel."""
    return np.bincount(pix, weights=valid, minlength=npix).round().astype(np.int64)


def pixel_matrices(pix, c, s, valid, kinds, comps, npix):
    """M_p = sum over samples t on pixel p and outputs o of v(t) w_o(t) w_o(t)^T.

    The normal matrix of the per-pixel map solve: the hitmap times the identity
    for a q+u polarimeter, the [3, 3] matrix of the IQU case (Sect. 3).
    """
    n_c = len(comps)
    n_t = pix.shape[0]
    M = np.zeros((npix, n_c, n_c))
    for kind in kinds:
        w = row_coefficients(kind, comps, c, s)
        for i, wi in w.items():
            for j, wj in w.items():
                prod = valid * _as_array(wi, n_t) * _as_array(wj, n_t)
                M[:, i, j] += np.bincount(pix, weights=prod, minlength=npix)
    return M


def pixel_cut(M, hits, rcond_min):
    """rcond = lambda_min / lambda_max of each symmetric M_p; keep h_p > 0 and
    rcond >= rcond_min; M_p^-1 on kept pixels, 0 elsewhere."""
    npix, n_c, _ = M.shape
    lam = np.linalg.eigvalsh(M)  # ascending eigenvalues per pixel
    with np.errstate(divide="ignore", invalid="ignore"):
        rcond = np.where(lam[:, -1] > 0, lam[:, 0] / lam[:, -1], 0.0)
    mask = (hits > 0) & (rcond >= rcond_min)
    Minv = np.zeros_like(M)
    if mask.any():
        Minv[mask] = np.linalg.inv(M[mask])
    return Minv, mask, rcond


def make_plan(pix, c, s, valid, nside, kinds, baseline_len, rcond_min=1e-3,
              npix=None) -> OraclePlan:
    """Everything that depends on the pointing only: hits, M, the cut, M^-1.

    npix overrides the map size 12 nside^2, for pixel indices that have been
    renumbered 0..npix-1 (a subset of the samples that holds every sample of the
    pixels it touches has the same per-pixel quantities as the whole problem)."""
    pix = np.asarray(pix, dtype=np.int64)
    n_t = pix.shape[0]
    npix = 12 * nside * nside if npix is None else int(npix)
    if n_t and (pix.min() < 0 or pix.max() >= npix):
        raise ValueError("pixel index out of range")
    c = np.asarray(c, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    valid = np.ones(n_t) if valid is None else np.asarray(valid, dtype=np.float64)
    kinds = tuple(kinds)
    comps = components(kinds)
    h = hitmap(pix, valid, npix)
    M = pixel_matrices(pix, c, s, valid, kinds, comps, npix)
    Minv, mask, rcond = pixel_cut(M, h, rcond_min)
    v = valid * mask[pix]
    n_b = -(-n_t // baseline_len)
    return OraclePlan(n_t, npix, kinds, comps, baseline_len, n_b, pix, c, s, valid, h, M,
                      rcond, mask, Minv, v)


def expand(plan: OraclePlan, x):
    """F~ x (Sect. 3, Eq. noise): baseline b repeated over its samples."""
    x = np.asarray(x, dtype=np.float64).reshape(plan.n_o, plan.n_b)
    return x[:, np.arange(plan.n_t) // plan.L]


def pixel_sums(plan: OraclePlan, z):
    """s_p = sum_t sum_o v w_o(t) z_o(t) per component and pixel: the binning
    P~^T R^T V of Sect. 3 before the pixel weight.  z is [n_o, n_t]; returns
    [n_c, npix]."""
    z = np.asarray(z, dtype=np.float64)
    summap = np.zeros((plan.n_c, plan.npix))
    for o, kind in enumerate(plan.kinds):
        w = row_coefficients(kind, plan.comps, plan.c, plan.s)
        for i, wi in w.items():
            summap[i] += np.bincount(plan.pix, weights=plan.v * _as_array(wi, plan.n_t) * z[o],
                                     minlength=plan.npix)
    return summap


def pixel_solve(plan: OraclePlan, summap):
    """m_p = M_p^-1 s_p on kept pixels, 0 on cut pixels (Eqs. mapQ/mapU with the
    general pixel weight)."""
    m = np.einsum("pij,jp->ip", plan.Minv, summap)
    m[:, ~plan.mask] = 0.0
    return m


def bin_map(plan: OraclePlan, z):
    """m = M^-1 sum_t sum_o v w_o(t) z_o(t), the ML map of Eqs. mapQ/mapU with the
    general pixel weight; 0 on cut pixels.  z is [n_o, n_t]."""
    return pixel_solve(plan, pixel_sums(plan, z))


def rescan(plan: OraclePlan, m):
    """A_p m: the map scanned back to every output's timeline (R P~ in Sect. 3)."""
    out = np.zeros((plan.n_o, plan.n_t))
    for o, kind in enumerate(plan.kinds):
        w = row_coefficients(kind, plan.comps, plan.c, plan.s)
        for i, wi in w.items():
            out[o] += _as_array(wi, plan.n_t) * m[i, plan.pix]
    return out


def baseline_sums(plan: OraclePlan, r):
    """F~^T r: sum of each output's timeline over every baseline period."""
    b = np.arange(plan.n_t) // plan.L
    return np.stack([np.bincount(b, weights=r[o], minlength=plan.n_b) for o in range(plan.n_o)])


def apply_Z(plan: OraclePlan, z):
    """Z z = V (z - A_p m(z)): the signal estimated from z is removed (Sect. 3)."""
    return plan.v * (z - rescan(plan, bin_map(plan, z)))


def apply_A(plan: OraclePlan, x):
    """Left-hand side of the destriping equation, F~^T (I - R P~ B) F~ x (Sect. 3)."""
    return baseline_sums(plan, apply_Z(plan, expand(plan, x))).reshape(-1)


def rhs(plan: OraclePlan, y):
    """Right-hand side of the destriping equation, F~^T (I - R P~ B) y (Sect. 3)."""
    return baseline_sums(plan, apply_Z(plan, y)).reshape(-1)


def cg(plan: OraclePlan, b, tol=1e-10, max_iter=10000, x0=None):
    """Conjugate gradient on A a = b (Sect. 3 names CG; A is symmetric PSD).

    Returns (x, iterations, ||r||/||b|| history).  Stops on the recursive residual.
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(plan, x) if x0 is not None else b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = float(np.sqrt(b @ b))
    hist = [np.sqrt(rr) / bnorm if bnorm > 0 else 0.0]
    it = 0
    if bnorm == 0.0:
        return x, 0, hist
    while it < max_iter and np.sqrt(rr) / bnorm >= tol:
        q = apply_A(plan, p)
        pq = float(p @ q)
        if pq <= 0.0:
            break
        alpha = rr / pq
        x += alpha * p
        r -= alpha * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        hist.append(np.sqrt(rr) / bnorm)
    return x, it, hist


def baseline_has_data(plan: OraclePlan):
    """[n_b] bool: the baseline holds at least one sample with v = 1."""
    b = np.arange(plan.n_t) // plan.L
    return np.bincount(b, weights=plan.v, minlength=plan.n_b) > 0


def gauge(plan: OraclePlan, a):
    """Fix the I null mode: remove, from the baselines of every output that carries
    I, their common mean over baselines with data; zero empty baselines."""
    a = np.array(a, dtype=np.float64).reshape(plan.n_o, plan.n_b)
    has = baseline_has_data(plan)
    a[:, ~has] = 0.0
    i_outs = [o for o, k in enumerate(plan.kinds) if k in ("I", "iqu")]
    if i_outs and has.any():
        mean = a[i_outs][:, has].mean()
        for o in i_outs:
            a[o, has] -= mean
    return a.reshape(-1)


def destripe(plan: OraclePlan, y, tol=1e-10, max_iter=10000):
    """Full method: RHS, CG for the baselines, gauge, destriped and binned maps
    (the outputs listed in Sect. 4: hitmap, binned map, destriped map, baselines)."""
    y = np.asarray(y, dtype=np.float64).reshape(plan.n_o, plan.n_t)
    b = rhs(plan, y)
    a, iters, hist = cg(plan, b, tol, max_iter)
    a = gauge(plan, a)
    dmap = bin_map(plan, y - expand(plan, a))
    bmap = bin_map(plan, y)
    return dict(a=a, map=dmap, binned=bmap, hits=plan.hits, mask=plan.mask, iters=iters,
                hist=hist, b=b)
