"""Host restatements of the two-level preconditioner's building blocks, checked
against their definitions (no GPU):

  * the coarse cells: every HEALPix RING pixel falls in exactly one of the
    12 nc^2 cells, every cell is hit, and a cell is a compact patch of sky;
  * the sweep operator with skipped pivots gives the inverse of an SPD matrix and
    a generalised inverse (E G E = E) of a singular positive semi-definite one;
  * the warp's segmented sum leaves, in the first lane of every run of equal
    consecutive keys, the sum of that run, also when a key comes back later.

Each restates the CUDA code's steps in numpy; a dropped shift, a wrong ring
offset, a pivot not skipped or a segment merged across a boundary fails one of
these checks.
"""
import math

import numpy as np
import pytest
import torch

from synth.healpix import ang2pix_ring


def isqrt(x):
    r = int(math.isqrt(int(x)))
    return r


def coarse_cell(p, N, nc):
    """Restatement of coarse_cell (precond.cu)."""
    npix, ncap = 12 * N * N, 2 * N * (N - 1)
    if p < ncap:
        i = (1 + isqrt(1 + 2 * p)) >> 1
        j = p - 2 * i * (i - 1)
        nring, ts = 4 * i, 1
    elif p < npix - ncap:
        q = p - ncap
        i = q // (4 * N) + N
        j = q - (i - N) * 4 * N
        nring, ts = 4 * N, (i - N + 1) & 1
    else:
        q = npix - 1 - p
        ii = (1 + isqrt(1 + 2 * q)) >> 1
        i = 4 * N - ii
        j = 4 * ii - 1 - (q - 2 * ii * (ii - 1))
        nring, ts = 4 * ii, 1
    k = min(max((2 * i * nc + N) // (2 * N), 1), 4 * nc - 1)
    if k < nc:
        nk, off = 4 * k, 2 * k * (k - 1)
    elif k <= 3 * nc:
        nk, off = 4 * nc, 2 * nc * (nc - 1) + (k - nc) * 4 * nc
    else:
        kk = 4 * nc - k
        nk, off = 4 * kk, 12 * nc * nc - 2 * kk * (kk + 1)
    return off + min(((2 * j + ts) * nk) // (2 * nring), nk - 1)


def ring_centres(N):
    """Pixel centres of the RING grid (colatitude, longitude) ring by ring."""
    th, ph = [], []
    for i in range(1, 4 * N):
        if i < N:
            n, z, s = 4 * i, 1 - i * i / (3 * N * N), 0.5
        elif i <= 3 * N:
            n, z, s = 4 * N, 4 / 3 - 2 * i / (3 * N), 0.5 * ((i - N + 1) % 2)
        else:
            ii = 4 * N - i
            n, z, s = 4 * ii, -(1 - ii * ii / (3 * N * N)), 0.5
        j = np.arange(n)
        th.append(np.full(n, math.acos(z)))
        ph.append((j + s) * 2 * math.pi / n)
    return np.concatenate(th), np.concatenate(ph)


@pytest.mark.parametrize("N,nc", [(16, 4), (32, 8), (64, 4), (8, 8), (128, 8)])
def test_coarse_cells_partition_the_sphere_into_compact_patches(N, nc):
    th, ph = ring_centres(N)
    # the centres are the RING grid's (they map back to their own index)
    assert np.array_equal(ang2pix_ring(N, torch.from_numpy(th), torch.from_numpy(ph)).numpy(),
                          np.arange(12 * N * N))
    cells = np.array([coarse_cell(p, N, nc) for p in range(12 * N * N)])
    assert cells.min() == 0 and cells.max() == 12 * nc * nc - 1
    assert len(np.unique(cells)) == 12 * nc * nc  # every cell holds pixels
    # compactness: every pixel lies within 2.5 cell sizes of its cell's mean direction
    v = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    cell_size = math.sqrt(4 * math.pi / (12 * nc * nc))
    for c in range(12 * nc * nc):
        sel = v[cells == c]
        m = sel.mean(0)
        m /= np.linalg.norm(m)
        ang = np.arccos(np.clip(sel @ m, -1, 1))
        assert ang.max() < 2.5 * cell_size, (c, ang.max(), cell_size)
    # a fine grid of a coarse grid's own resolution maps one pixel per cell
    if N == nc:
        assert np.array_equal(np.sort(cells), np.arange(12 * N * N))


def sweep_inverse(E, tol_rel=1e-10):
    """Restatement of the sweep steps (k_pc_sweep, k_pc_finish)."""
    A = E.astype(np.float64).copy()
    n = A.shape[0]
    d0 = np.diag(A).copy()
    skipped = np.zeros(n, bool)
    for k in range(n):
        d = A[k, k]
        if not d > tol_rel * d0[k]:
            skipped[k] = True
            continue
        out = A - np.outer(A[:, k], A[k, :]) / d
        out[k, :] = A[k, :] / d
        out[:, k] = A[:, k] / d
        out[k, k] = -1.0 / d
        A = out
    G = -A
    G[skipped, :] = 0.0
    G[:, skipped] = 0.0
    return G, skipped


def test_sweep_inverts_spd_matrix():
    rng = np.random.default_rng(1)
    B = rng.standard_normal((40, 40))
    E = B @ B.T + 0.1 * np.eye(40)
    G, skipped = sweep_inverse(E)
    assert not skipped.any()
    assert np.allclose(G, np.linalg.inv(E), rtol=1e-8, atol=1e-10)


def test_sweep_gives_generalised_inverse_of_singular_psd():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((30, 22))
    E = B @ B.T  # rank 22
    G, skipped = sweep_inverse(E)
    assert skipped.sum() == 8
    assert np.allclose(E @ G @ E, E, rtol=1e-7, atol=1e-7 * np.abs(E).max())
    assert np.allclose(G, G.T)
    # positive semi-definite: a valid part of an SPD preconditioner
    assert np.linalg.eigvalsh(G).min() > -1e-8 * np.abs(G).max()


def test_sweep_with_null_mode_and_rank_one_term():
    # a matrix whose null vector is the indicator u of some columns, made definite by
    # the rank-one term mu u u^T / |u|^2 (the I gauge of the coarse matrix)
    rng = np.random.default_rng(3)
    n, m = 24, 8
    u = np.zeros(n)
    u[:m] = 1.0
    P = np.eye(n) - np.outer(u, u) / m
    B = rng.standard_normal((n, n))
    E = P @ (B @ B.T) @ P
    mu = np.trace(E) / n
    Er = E + mu * np.outer(u, u) / m
    G, skipped = sweep_inverse(Er)
    assert not skipped.any()
    assert np.allclose(G @ Er, np.eye(n), atol=1e-8)
    # on vectors orthogonal to u the term changes nothing
    x = P @ rng.standard_normal(n)
    assert np.allclose(Er @ x, E @ x)


def seg_sum_to_head(keys, vals):
    """Restatement of seg_sum_to_head (cg.cu): doubling steps over a warp of 32."""
    keys = np.asarray(keys)
    v = np.asarray(vals, dtype=np.float64).copy()
    stop = np.array([l == 31 or keys[l + 1] != keys[l] for l in range(32)])
    w = 1
    while w < 32:
        v2 = np.array([v[l + w] if l + w < 32 else v[l] for l in range(32)])
        s2 = np.array([stop[l + w] if l + w < 32 else stop[l] for l in range(32)])
        add = ~stop
        v = np.where(add, v + v2, v)
        stop = np.where(add, s2, stop)
        w <<= 1
    return v


@pytest.mark.parametrize("seed", range(20))
def test_segmented_sum_reaches_each_segment_head(seed):
    rng = np.random.default_rng(seed)
    # runs of equal keys, keys drawn from a few values so that they come back
    keys = np.repeat(rng.integers(-1, 4, 32), rng.integers(1, 6, 32))[:32]
    vals = rng.standard_normal(32)
    got = seg_sum_to_head(keys, vals)
    l = 0
    while l < 32:
        e = l
        while e + 1 < 32 and keys[e + 1] == keys[l]:
            e += 1
        assert abs(got[l] - vals[l:e + 1].sum()) < 1e-12
        l = e + 1


def warp_buffered_terms(pixels, nE, nc, max_cells=8):
    """Host restatement of the coarse matrix's per-warp buffer (k_pc_E_*): each
    pixel's term over its cells is added into a buffer over at most max_cells
    cells; new cells are appended while there is room, else the buffer is added
    into E and restarts with the pixel's cells.  pixels: [(cells, term)] with
    term an (len(cells) nc) x (len(cells) nc) block."""
    E = np.zeros((nE, nE))
    ids, buf = [], np.zeros((max_cells * nc, max_cells * nc))
    stale = list(range(1000, 1000 + max_cells))  # ids of slots not in use

    def flush():
        m = len(ids) * nc
        for e1 in range(m):
            for e2 in range(m):
                E[ids[e1 // nc] * nc + e1 % nc, ids[e2 // nc] * nc + e2 % nc] += buf[e1, e2]
        buf[:] = 0.0

    for cells, term in pixels:
        slots, n0, nb = [], len(ids), len(ids)
        for c in cells:  # search the buffer's cells only, never the stale slots
            idx = ids.index(c) if c in ids[:n0] else -1
            if idx < 0:
                idx = nb if nb < max_cells else -1
                nb += 1
            slots.append(idx)
        if nb > max_cells:
            flush()
            ids, slots = list(cells), list(range(len(cells)))
        else:
            for c, s in zip(cells, slots):
                if s >= len(ids):
                    ids.append(c)
        for i, s1 in enumerate(slots):
            for j, s2 in enumerate(slots):
                buf[s1 * nc:(s1 + 1) * nc, s2 * nc:(s2 + 1) * nc] += term[i * nc:(i + 1) * nc,
                                                                           j * nc:(j + 1) * nc]
    flush()
    return E


def test_warp_buffer_of_pixel_terms_equals_direct_sum():
    rng = np.random.default_rng(7)
    ncell, nc = 40, 3
    pixels, cur = [], [0]
    for _ in range(2000):  # neighbouring pixels mostly share cells
        if rng.random() < 0.3:
            cur = sorted(set(int(c) for c in rng.integers(0, ncell, size=rng.integers(1, 5))))
        cells = list(cur)
        rng.shuffle(cells)
        k = len(cells) * nc
        pixels.append((cells, rng.standard_normal((k, k))))
    direct = np.zeros((ncell * nc, ncell * nc))
    for cells, term in pixels:
        for i, c1 in enumerate(cells):
            for j, c2 in enumerate(cells):
                direct[c1 * nc:(c1 + 1) * nc, c2 * nc:(c2 + 1) * nc] += term[i * nc:(i + 1) * nc,
                                                                           j * nc:(j + 1) * nc]
    got = warp_buffered_terms(pixels, ncell * nc, nc)
    assert np.allclose(got, direct, rtol=0, atol=1e-9)
