"""Dense brute-force form of the destriping system, for tiny problems only.

TEST INFRASTRUCTURE ONLY (see oracle/core.py).

Builds every matrix of Sect. 3 explicitly -- F~ [n_o n_t, n_o n_b], the pointing
and rotation operator A_p [n_o n_t, n_c n_pix], the weights V -- and forms

    A = F~^T (V - V A_p (A_p^T V A_p)^+ A_p^T V) F~,   b = F~^T (V - ...) y

with a pseudo-inverse, so it shares no step with the matrix-free oracle except
the row definitions.  The pixel cut is recomputed here from the dense normal
matrix blocks.
"""
from __future__ import annotations

import numpy as np

from .core import components, row_coefficients


def dense_system(pix, c, s, valid, nside, kinds, L, rcond_min=1e-3):
    pix = np.asarray(pix, dtype=np.int64)
    n_t = pix.shape[0]
    npix = 12 * nside * nside
    kinds = tuple(kinds)
    comps = components(kinds)
    n_o, n_c = len(kinds), len(comps)
    n_b = -(-n_t // L)
    c = np.asarray(c, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    val = np.ones(n_t) if valid is None else np.asarray(valid, dtype=np.float64)
    F = np.zeros((n_o * n_t, n_o * n_b))
    Ap = np.zeros((n_o * n_t, n_c * npix))
    for o, kind in enumerate(kinds):
        for t in range(n_t):
            F[o * n_t + t, o * n_b + t // L] = 1.0
        w = row_coefficients(kind, comps, c, s)
        for i, wi in w.items():
            coef = np.full(n_t, wi) if np.isscalar(wi) else wi
            Ap[o * n_t + np.arange(n_t), i * npix + pix] = coef
    Vin = np.diag(np.tile(val, n_o))
    G = Ap.T @ Vin @ Ap
    # per-pixel blocks of G: indices (i * npix + p) for i in components
    keep = np.zeros(npix, dtype=bool)
    for p in range(npix):
        idx = [i * npix + p for i in range(n_c)]
        blk = G[np.ix_(idx, idx)]
        lam = np.linalg.eigvalsh(blk)
        keep[p] = lam[-1] > 0 and lam[0] / lam[-1] >= rcond_min and val[pix == p].sum() > 0
    v = val * keep[pix]
    V = np.diag(np.tile(v, n_o))
    Z = V - V @ Ap @ np.linalg.pinv(Ap.T @ V @ Ap) @ Ap.T @ V
    A = F.T @ Z @ F
    return dict(A=A, Z=Z, F=F, Ap=Ap, V=V, keep=keep, n_b=n_b, n_c=n_c, npix=npix)


def dense_solve(pix, c, s, valid, nside, kinds, L, y, rcond_min=1e-3):
    """Min-norm solution of the destriping equation by pseudo-inverse."""
    d = dense_system(pix, c, s, valid, nside, kinds, L, rcond_min)
    yv = np.asarray(y, dtype=np.float64).reshape(-1)
    b = d["F"].T @ d["Z"] @ yv
    a = np.linalg.pinv(d["A"], rcond=1e-10) @ b
    return a, b, d
