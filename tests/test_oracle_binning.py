"""Pins of the tile-binning reference (the integer stage of the rasterizer; the paper
says only that Gaussians are "projected and rasterized", Sec. 3.1): hand-worked cases,
brute force over (Gaussian, tile) pairs, the FP64 rule, and the stable sort of keys."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "binning_cases.txt")


def load_cases():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b = line.split("|")
        u, v, ex, ey, W, H, TW, TH = a.split()
        rows.append(((float(u), float(v), float(ex), float(ey), int(W), int(H), int(TW), int(TH)),
                     tuple(int(x) for x in b.split())))
    return rows


def test_hand_worked_cases():
    cases = load_cases()
    assert len(cases) >= 9
    for (u, v, ex, ey, W, H, TW, TH), expect in cases:
        cnt, rect = oracle.bin_f32([u], [v], [ex], [ey], [1], W, H, TW, TH)
        assert (cnt[0], *rect[0]) == expect, (u, v, ex, ey, expect, cnt, rect)
        c64, r64, _ = oracle.bin_f64([u], [v], [ex], [ey], [1], W, H, TW, TH)
        assert (c64[0], *r64[0]) == expect


def brute_force_counts(u, v, ex, ey, valid, W, H, TW, TH):
    """For each (Gaussian, tile): does any pixel centre of the tile lie in the extent box?"""
    xs = np.arange(W) + 0.5
    ys = np.arange(H) + 0.5
    counts = np.zeros(len(u), np.int64)
    tiles_x, tiles_y = (W + TW - 1) // TW, (H + TH - 1) // TH
    for i in range(len(u)):
        if not valid[i]:
            continue
        colx = (xs >= u[i] - ex[i]) & (xs <= u[i] + ex[i])
        coly = (ys >= v[i] - ey[i]) & (ys <= v[i] + ey[i])
        n = 0
        for ty in range(tiles_y):
            for tx in range(tiles_x):
                if colx[tx * TW:(tx + 1) * TW].any() and coly[ty * TH:(ty + 1) * TH].any():
                    n += 1
        counts[i] = n
    return counts


def test_counts_match_brute_force_on_dyadic_inputs():
    """Inputs on a 1/64 grid keep every FP32 operation of the rule exact, so the rule must
    agree exactly with real-arithmetic brute force, for every tile shape."""
    rng = np.random.default_rng(4)
    n = 400
    for (W, H) in ((96, 64), (100, 37)):
        u = np.round(rng.uniform(-20, W + 20, n) * 64) / 64
        v = np.round(rng.uniform(-20, H + 20, n) * 64) / 64
        ex = np.round(rng.exponential(6, n) * 64) / 64
        ey = np.round(rng.exponential(6, n) * 64) / 64
        valid = rng.uniform(size=n) > 0.1
        for TW, TH in ((8, 8), (16, 16), (16, 8)):
            cnt, rect = oracle.bin_f32(u, v, ex, ey, valid, W, H, TW, TH)
            bf = brute_force_counts(u, v, ex, ey, valid, W, H, TW, TH)
            assert np.array_equal(cnt, bf), (W, H, TW, TH)
            nz = cnt > 0
            assert np.array_equal(cnt[nz], (rect[nz, 2] - rect[nz, 0] + 1) * (rect[nz, 3] - rect[nz, 1] + 1))
            c64, r64, _ = oracle.bin_f64(u, v, ex, ey, valid, W, H, TW, TH)
            assert np.array_equal(c64, cnt) and np.array_equal(r64, rect)


def test_counts_match_brute_force_on_random_fp32_inputs():
    """Random FP32 inputs: agreement with brute force except where an extent edge lies
    within FP32 rounding of a pixel centre."""
    rng = np.random.default_rng(5)
    n = 500
    W, H = 120, 80
    u = rng.uniform(-10, W + 10, n).astype(np.float32)
    v = rng.uniform(-10, H + 10, n).astype(np.float32)
    ex = rng.exponential(5, n).astype(np.float32)
    ey = rng.exponential(5, n).astype(np.float32)
    valid = np.ones(n, bool)
    cnt, rect = oracle.bin_f32(u, v, ex, ey, valid, W, H, 16, 16)
    bf = brute_force_counts(u.astype(np.float64), v.astype(np.float64), ex.astype(np.float64),
                            ey.astype(np.float64), valid, W, H, 16, 16)
    _, _, margin = oracle.bin_f64(u, v, ex, ey, valid, W, H, 16, 16)
    bad = cnt != bf
    assert np.all(margin[bad] < 1e-4)
    assert bad.sum() <= 2


def test_sorted_keys_order_and_stability():
    """Emitted keys sorted by (tile, depth bits), ties (equal depth) in Gaussian order; the
    list is a permutation of the emitted one; ranges partition it."""
    rng = np.random.default_rng(6)
    n, W, H, TW, TH = 300, 64, 48, 16, 16
    u = rng.uniform(0, W, n).astype(np.float32)
    v = rng.uniform(0, H, n).astype(np.float32)
    ex = rng.exponential(8, n).astype(np.float32)
    ey = rng.exponential(8, n).astype(np.float32)
    depth = rng.choice(np.array([2.0, 3.5, 7.25], np.float32), n)  # many ties
    cnt, rect = oracle.bin_f32(u, v, ex, ey, np.ones(n, bool), W, H, TW, TH)
    keys, vals = oracle.emit_keys(cnt, rect, depth, (W + TW - 1) // TW)
    assert len(keys) == cnt.sum()
    sk, sv = oracle.sorted_keys(keys, vals)
    # textbook check: Python's sort of (key, emit position) tuples
    ref = sorted(range(len(keys)), key=lambda i: (int(keys[i]), i))
    assert np.array_equal(sv, vals[ref]) and np.array_equal(sk, keys[ref])
    tiles = (sk >> np.uint64(32)).astype(np.int64)
    for t in np.unique(tiles):
        seg = sv[tiles == t]
        d = depth[seg]
        assert np.all(np.diff(d) >= 0)
        same = np.diff(d) == 0
        assert np.all(np.diff(seg)[same] > 0)
    ranges = oracle.tile_ranges(sk, 12)
    assert ranges[0, 0] == 0 and ranges[-1, 1] == len(sk)
    assert np.all(ranges[1:, 0] == ranges[:-1, 1])
