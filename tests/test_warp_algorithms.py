"""Host restatements of the warp-level algorithms of the CUDA kernels, each checked
against the plain sequential definition on small random cases (ragged ends,
flags, baselines of 1 to 5000 samples).  They pin the designs (which lane
writes what, when a warp flushes, how offsets compose); the -m gpu tests check
the kernels themselves against the oracle.

  * run construction (runs_build.cu): per-block run counts in warp shares with a
    top-level scan, and the fill's rounds of 32 lanes: ballot of run starts,
    segmented scan limited to the longest run, runs carried across rounds;
  * carried baseline sums (k_rl_rescan, k_rl_rescan_df, k_rescan_df): per-lane sums
    kept across rounds, warp flushes only where a baseline ends;
  * run hand-off in the accurate binning (k_bin_df): a lane's last run carried
    into the next lane's first when they share a pixel;
  * the two-level offsets of the pixel-major copy (k_pm_scan_up / k_pm_scan_down);
  * the lane-sequential binning over pixel-sorted records (k_tl_bin_lanes): a lane's
    head, interior and tail pixels, the segmented scan of tails over the lanes, and
    the pixel carried across rounds: every pixel reduced once per chunk;
  * the fixed-point baseline sums of the tiled rescan (k_tl_rescan): the scale from
    the map maximum, the split into integer and fraction parts, no partial sum
    outside int32, and the sum recovered to half a unit per term."""
import math

import numpy as np
import pytest

LANES = 32


def run_starts(pix, L):
    n = len(pix)
    return [pix[t] >= 0 and (t % L == 0 or pix[t - 1] != pix[t]) for t in range(n)]


def runs_sequential(pix, c, L):
    """(pixel, count, sum c, baseline) of every run, in sample order."""
    out, t, n = [], 0, len(pix)
    st = run_starts(pix, L)
    while t < n:
        if st[t]:
            u, cnt, s = t, 0, 0.0
            while u < n and (u == t or u % L != 0) and pix[u] == pix[t]:
                cnt += 1
                s += c[u]
                u += 1
            out.append((int(pix[t]), cnt, s, t // L))
        t += 1
    return out


def count_split(n_sub, grid, warps_per_block=8):
    S = -(-n_sub // grid)
    G = -(-n_sub // S)
    return S, G, warps_per_block


def block_offsets(counts, grid):
    """k_rl_count's within-block offsets and k_rl_scan's block offsets."""
    n_sub = len(counts)
    S, G, W = count_split(n_sub, grid)
    sub_off = np.zeros(n_sub, dtype=np.int64)
    blk = np.zeros(G, dtype=np.int64)
    per = -(-S // W)
    for j in range(G):
        b0, b1 = j * S, min(j * S + S, n_sub)
        run, shares = 0, []
        for q in range(W):
            lo = min(b0 + q * per, b1)
            hi = min(lo + per, b1)
            wrun = 0
            for w in range(lo, hi):
                sub_off[w] = wrun
                wrun += counts[w]
            shares.append((lo, hi, run))
            run += wrun
        for lo, hi, wo in shares:
            sub_off[lo:hi] += wo
        blk[j] = run
    excl = np.concatenate([[0], np.cumsum(blk)[:-1]])
    return sub_off + excl[np.arange(n_sub) // S]


def fill(pix, c, L, ksub):
    n_t = len(pix)
    n_sub = -(-n_t // ksub)
    st = run_starts(pix, L)
    counts = [sum(st[w * ksub:min((w + 1) * ksub, n_t)]) for w in range(n_sub)]
    base_of = block_offsets(counts, grid=max(1, n_sub // 3))
    rec = [None] * sum(counts)
    for w in range(n_sub):
        base, cn, cs, cr = int(base_of[w]), 0, 0.0, -1
        t0 = w * ksub
        while True:
            own = t0 < (w + 1) * ksub
            if not own and cr < 0:
                break
            ts = [t0 + l for l in range(LANES)]
            p = [int(pix[t]) if t < n_t else -1 for t in ts]
            rstart = [t < n_t and st[t] for t in ts]
            smask = [own and r for r in rstart]
            head = [max([k for k in range(l + 1) if rstart[k]], default=-1) for l in range(LANES)]
            member = [p[l] >= 0 and (own if head[l] >= 0 else cr >= 0) for l in range(LANES)]
            n = [1 if m else 0 for m in member]
            s = [c[ts[l]] if member[l] else 0.0 for l in range(LANES)]
            seg0 = [h if h >= 0 else 0 for h in head]
            reach = max([l - seg0[l] for l in range(LANES) if member[l]], default=0)
            d = 1
            while d < LANES and d <= reach:   # segmented Hillis-Steele scan, limited steps
                n2, s2 = n[:], s[:]
                for l in range(LANES):
                    if l - d >= seg0[l]:
                        n2[l] += n[l - d]
                        s2[l] += s[l - d]
                n, s, d = n2, s2, d * 2
            for l in range(LANES):
                if head[l] < 0 and cr >= 0:
                    n[l] += cn
                    s[l] += cs
            conts = []
            for l in range(LANES):
                if l < LANES - 1:
                    cont = member[l + 1] and not smask[l + 1]
                else:
                    u = ts[l] + 1
                    cont = member[l] and u < n_t and u % L != 0 and pix[u] == p[l]
                conts.append(cont)
                r = base + sum(smask[:head[l]]) if head[l] >= 0 else cr
                if member[l] and not cont:
                    assert rec[r] is None
                    rec[r] = (p[l], n[l], s[l], ts[l] // L)
            r31 = base + sum(smask[:head[31]]) if head[31] >= 0 else cr
            carry = member[31] and conts[31]
            cn, cs, cr = n[31], s[31], (r31 if carry else -1)
            base += sum(smask)
            t0 += LANES
    return rec


def random_pointing(rng, n_t, npix=(2, 5, 50, 1000), flag=(0, 0.05, 0.3)):
    pix = []
    while len(pix) < n_t:
        pix += [int(rng.integers(0, int(rng.choice(npix))))] * int(
            rng.integers(1, int(rng.choice([2, 5, 40, 300]))))
    pix = np.array(pix[:n_t])
    pix[rng.random(n_t) < rng.choice(flag)] = -1
    return pix


def test_run_construction_matches_the_sequential_split():
    rng = np.random.default_rng(1)
    for trial in range(25):
        n_t = int(rng.integers(1, 1500))
        L = int(rng.choice([1, 3, 31, 32, 33, 97, 5000]))
        pix = random_pointing(rng, n_t)
        c = rng.integers(-8, 9, n_t).astype(float)
        ref = runs_sequential(pix, c, L)
        got = fill(pix, c, L, ksub=int(rng.choice([64, 128])))
        assert got == [(p, n, s, b) for p, n, s, b in ref], (trial, n_t, L)


def test_block_offsets_are_the_exclusive_prefix():
    rng = np.random.default_rng(2)
    for n_sub in (1, 2, 7, 8, 9, 100, 1217, 5000):
        for grid in (1, 3, 152 * 8):
            counts = rng.integers(0, 50, n_sub)
            want = np.concatenate([[0], np.cumsum(counts)[:-1]])
            assert (block_offsets(counts, min(grid, n_sub)) == want).all()


def segmented_flush(keys, vals, out):
    """The warp's segmented sum over lanes (equal keys must be contiguous)."""
    seen = {}
    for l, k in enumerate(keys):
        if k >= 0:
            assert k not in seen or seen[k] == l - 1, keys
            seen[k] = l
    v = list(vals)
    d = 1
    while d < LANES:
        v = [v[l] + (v[l + d] if l + d < LANES and keys[l + d] == keys[l] else 0)
             for l in range(LANES)]
        d *= 2
    for l in range(LANES):
        if keys[l] >= 0 and (l == 0 or keys[l - 1] != keys[l]):
            out[keys[l]] += v[l]


def carried_rescan(valid, val, xterm, L, rounds):
    """k_rescan_df's chunks of `rounds` x 128 samples, 4 per lane per round."""
    n_t = len(val)
    nvec = -(-n_t // 4)
    span = rounds * LANES
    out = np.zeros(-(-n_t // L))
    for ch in range(-(-nvec // span)):
        key, cnt, acc = [-1] * LANES, [0] * LANES, [0.0] * LANES

        def fold(l):
            if key[l] >= 0 and cnt[l]:
                acc[l] += cnt[l] * xterm[key[l]]

        for r in range(rounds):
            v = [ch * span + r * LANES + l for l in range(LANES)]
            active = [x < nvec for x in v]
            if not any(active):
                break
            bf = [4 * x // L for x in v]
            if any(not active[l] or (key[l] >= 0 and bf[l] != key[l]) for l in range(LANES)):
                for l in range(LANES):
                    fold(l)
                segmented_flush(key, acc, out)
                key, cnt, acc = [-1] * LANES, [0] * LANES, [0.0] * LANES
            for l in range(LANES):
                if not active[l]:
                    continue
                if key[l] < 0:
                    key[l] = bf[l]
                t0 = 4 * v[l]
                bend = (t0 // L + 1) * L
                for t in range(t0, min(t0 + 4, n_t)):
                    if t >= bend:   # the lane's samples cross a baseline end
                        fold(l)
                        out[key[l]] += acc[l]
                        key[l], cnt[l], acc[l] = key[l] + 1, 0, 0.0
                        bend += L
                    if valid[t]:
                        cnt[l] += 1
                        acc[l] += val[t]
        for l in range(LANES):
            fold(l)
        segmented_flush(key, acc, out)
    return out


@pytest.mark.parametrize("rounds", [1, 3, 16])
def test_carried_baseline_sums_reach_every_baseline_once(rounds):
    rng = np.random.default_rng(3 + rounds)
    for trial in range(12):
        n_t = int(rng.integers(1, 5000))
        L = int(rng.choice([1, 2, 3, 5, 64, 127, 128, 129, 3000, 10 ** 6]))
        valid = rng.random(n_t) > rng.choice([0, 0.1, 0.6])
        val = rng.integers(-5, 6, n_t).astype(float)
        xterm = rng.integers(-3, 4, -(-n_t // L)).astype(float)
        want = np.zeros_like(xterm)
        for t in range(n_t):
            if valid[t]:
                want[t // L] += val[t] + xterm[t // L]
        assert np.array_equal(carried_rescan(valid, val, xterm, L, rounds), want), (n_t, L)


def handoff_flushes(pix4, val4):
    """k_bin_df: per lane 4 samples; first and last runs stay open, the last runs
    flow right through a segmented scan while pixels match."""
    fl = []
    head_p, tail_p = [-1] * LANES, [-1] * LANES
    head, tail, nruns = [0.0] * LANES, [0.0] * LANES, [0] * LANES
    for l in range(LANES):
        cur, acc = -1, 0.0
        for p, v in zip(pix4[l], val4[l]):
            if p < 0:
                continue
            if p != cur:
                if cur >= 0:
                    if nruns[l] == 1:
                        head_p[l], head[l] = cur, acc
                    else:
                        fl.append((cur, acc))
                cur, acc = p, 0.0
                nruns[l] += 1
            acc += v
        tail_p[l], tail[l] = cur, acc
        if nruns[l] == 1:
            head_p[l] = cur
    single = [k == 1 for k in nruns]
    link = [l > 0 and head_p[l] >= 0 and head_p[l] == tail_p[l - 1] for l in range(LANES)]
    through = [single[l] and link[l] for l in range(LANES)]
    seg0 = [max(k for k in range(l + 1) if not through[k]) for l in range(LANES)]
    out, d = list(tail), 1
    while d < LANES:
        out = [out[l] + (out[l - d] if l - d >= seg0[l] else 0.0) for l in range(LANES)]
        d *= 2
    for l in range(LANES):
        nxt = l < LANES - 1 and link[l + 1]
        if not single[l] and head_p[l] >= 0:
            fl.append((head_p[l], head[l] + (out[l - 1] if link[l] else 0.0)))
        if tail_p[l] >= 0 and not nxt:
            fl.append((tail_p[l], out[l] if single[l] else tail[l]))
    return fl


def test_run_handoff_bins_every_sample_once_with_fewer_flushes():
    rng = np.random.default_rng(7)
    n_plain = n_hand = 0
    for trial in range(400):
        pix = random_pointing(rng, 128, npix=(3, 50, 10 ** 6), flag=(0, 0.05, 0.5))
        if rng.random() < 0.1:
            pix[rng.integers(0, 128):] = -1
        val = rng.integers(-9, 10, 128).astype(float)
        fl = handoff_flushes(pix.reshape(LANES, 4).tolist(), val.reshape(LANES, 4).tolist())
        want, got = {}, {}
        for p, v in zip(pix, val):
            if p >= 0:
                want[p] = want.get(p, 0.0) + v
        for p, v in fl:
            got[p] = got.get(p, 0.0) + v
        assert want == got, trial
        n_hand += len(fl)
        n_plain += sum(len([k for k in range(4) if g[k] >= 0 and (k == 0 or g[k] != g[k - 1]
                                                                      or g[k - 1] < 0)])
                       for g in pix.reshape(LANES, 4).tolist())
    assert n_hand < n_plain


def test_pixel_major_offsets_are_the_exclusive_prefix_of_runs_per_pixel():
    rng = np.random.default_rng(9)
    for npix in (1, 7, 256, 257, 5000):
        cnt = rng.integers(0, 70, npix)
        grid = max(1, min(npix, 37))
        S = -(-npix // grid)
        G = -(-npix // S)
        blk = np.array([cnt[j * S:min(npix, (j + 1) * S)].sum() for j in range(G)])
        excl = np.concatenate([[0], np.cumsum(blk)[:-1]])
        off = np.empty(npix + 1, dtype=np.int64)
        for j in range(G):   # tiles of 256 pixels, a carried prefix within the block
            carry = excl[j]
            for base in range(j * S, min(npix, (j + 1) * S), 256):
                tile = cnt[base:min(base + 256, (j + 1) * S, npix)]
                off[base:base + len(tile)] = carry + np.cumsum(tile) - tile
                carry += tile.sum()
        off[npix] = cnt.sum()
        assert (off == np.concatenate([[0], np.cumsum(cnt)])).all()


# ---- lane-sequential binning over pixel-sorted records (k_tl_bin_lanes) --------------

LANE_RECS = 8
ROUND = LANES * LANE_RECS


def lanes_round_flushes(keys, vals, ckey, carry):
    """One round of k_tl_bin_lanes: keys/vals of the round's ROUND records (key -1
    past the chunk's end, only at the end), the pixel carried from the previous
    round.  Returns (flushes [(key, value)], new ckey, new carry)."""
    flushes = []
    cur = [-1] * LANES
    hkey = [-1] * LANES
    head = [False] * LANES
    acc = [0.0] * LANES
    hacc = [0.0] * LANES
    for l in range(LANES):  # each lane sums its LANE_RECS consecutive records
        for k in range(LANE_RECS):
            key, w = keys[l * LANE_RECS + k], vals[l * LANE_RECS + k]
            if key < 0:
                continue
            if key != cur[l]:
                if cur[l] >= 0:
                    if not head[l]:
                        head[l], hkey[l], hacc[l] = True, cur[l], acc[l]
                    else:
                        flushes.append((cur[l], acc[l]))  # interior pixel
                cur[l], acc[l] = key, w
            else:
                acc[l] += w
    first = [hkey[l] if head[l] else cur[l] for l in range(LANES)]
    if ckey >= 0:  # the carried pixel joins lane 0's first pixel, or is complete
        if first[0] == ckey:
            if head[0]:
                hacc[0] += carry
            else:
                acc[0] += carry
        else:
            flushes.append((ckey, carry))
    prev = [cur[0]] + cur[:-1]  # shfl_up by one: lane 0 reads itself
    f = [l == 0 or head[l] or prev[l] != cur[l] for l in range(LANES)]
    s = list(acc)
    d = 1
    while d < LANES:  # Hillis-Steele segmented inclusive scan of the tails
        s_up, f_up = list(s), list(f)
        for l in range(LANES):
            if l >= d and not f[l]:
                s_up[l] = s[l] + s[l - d]
                f_up[l] = f[l - d]
            else:
                s_up[l], f_up[l] = s[l], f[l]
        s, f = s_up, f_up
        d *= 2
    for l in range(LANES):
        if head[l]:
            v = hacc[l] + (s[l - 1] if l > 0 and prev[l] == hkey[l] else 0.0)
            flushes.append((hkey[l], v))
    nxt = first[1:] + [first[-1]]
    for l in range(LANES - 1):
        if cur[l] >= 0 and nxt[l] != cur[l]:
            flushes.append((cur[l], s[l]))
    return flushes, cur[LANES - 1], s[LANES - 1]


def lanes_chunk_flushes(keys, vals):
    flushes, ckey, carry = [], -1, 0.0
    for base in range(0, len(keys), ROUND):
        k = list(keys[base:base + ROUND]) + [-1] * max(0, base + ROUND - len(keys))
        v = list(vals[base:base + ROUND]) + [0.0] * max(0, base + ROUND - len(vals))
        fl, ckey, carry = lanes_round_flushes(k, v, ckey, carry)
        flushes += fl
    if ckey >= 0:
        flushes.append((ckey, carry))
    return flushes


@pytest.mark.parametrize("mean_run", [1.0, 1.5, 7.0, 40.0, 600.0])
def test_lane_sequential_binning_sums_every_pixel_once_per_chunk(mean_run):
    rng = np.random.default_rng(int(mean_run * 10))
    for n in (1, 7, ROUND - 1, ROUND, ROUND + 1, 5 * ROUND + 123):
        # pixel-sorted keys: segments of geometric length
        keys = []
        p = 0
        while len(keys) < n:
            p += int(rng.integers(1, 4))
            keys += [p] * int(rng.geometric(1.0 / mean_run))
        keys = keys[:n]
        vals = rng.integers(-8, 9, size=n).astype(float)  # exact sums in any order
        flushes = lanes_chunk_flushes(keys, vals)
        got, seen = {}, {}
        for k, v in flushes:
            got[k] = got.get(k, 0.0) + v
            seen[k] = seen.get(k, 0) + 1
        want = {}
        for k, v in zip(keys, vals):
            want[k] = want.get(k, 0.0) + v
        assert got == want
        # one flush per pixel: a pixel's records are contiguous within the chunk
        assert all(c == 1 for c in seen.values()), seen


# ---- fixed-point baseline sums of the tiled rescan (k_tl_rescan) ---------------------

def fixed_point_scale(L, big):
    """The rescan's exponents: e with L x 3 x big x 2^e <= 2^30, f fraction bits."""
    e = 0
    if big > 0.0:
        _, ex = math.frexp(L * 3.0 * big)
        e = min(126, max(-126, 30 - ex))
    f = min(16, max(0, 30 - int(L).bit_length()))
    return e, f


@pytest.mark.parametrize("L,big", [(1, 1.0), (50, 37.5), (50, 1e-20), (3000, 2.5e6), (30000, 0.3),
                                   (200000, 5.0)])
def test_fixed_point_baseline_sums_match_float64(L, big):
    rng = np.random.default_rng(L)
    e, f = fixed_point_scale(L, big)
    scale, frac = np.float32(2.0 ** e), np.float32(2.0 ** f)
    for trial in range(20):
        # one baseline: runs of n samples (sum n <= L), terms up to n x 3 x big
        n = []
        while sum(n) < L:
            n.append(int(min(L - sum(n), rng.integers(1, 256))))
        n = np.array(n)
        terms = (rng.uniform(-1.0, 1.0, size=len(n)) * n * 3.0 * big).astype(np.float32)
        if trial == 0:
            terms = (n * 3.0 * big * np.sign(rng.uniform(-1, 1))).astype(np.float32)  # the bound
        v = terms * scale  # exact: a power of two
        h = np.rint(v)
        lo = np.rint((v - h) * frac)
        assert np.all((v - h) == (v.astype(np.float64) - h.astype(np.float64)))  # exact rest
        hi_sum = np.cumsum(h.astype(np.int64))
        lo_sum = np.cumsum(lo.astype(np.int64))
        assert np.abs(hi_sum).max() < 2 ** 31 and np.abs(lo_sum).max() < 2 ** 31
        got = float(hi_sum[-1]) * 2.0 ** -e + float(lo_sum[-1]) * 2.0 ** (-e - f)
        want = float(np.sum(terms.astype(np.float64)))
        # each term is kept to half a unit of 2^-(e + f); the float32 terms are the input
        assert abs(got - want) <= len(n) * 0.5 * 2.0 ** (-e - f) * (1 + 1e-9) + 1e-300
