"""Pins of the culled tile-binning rule (the integer stage of the rasterizer; Sec. 3.1 of
the paper only says that Gaussians are "projected and rasterized"): a Gaussian is binned
into the tiles of its extent box whose band of pixel-centre rows reaches its
alpha >= 1/255 ellipse d^T Sigma2^{-1} d <= tau.  Pinned by hand-worked cases, by FP64
brute force over pixel centres (no pixel centre inside the ellipse is ever left out, and
every kept tile has a pixel column that reaches the ellipse inside its band), and by the
stable order of the emitted keys."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "binning_cull_cases.txt")
TILES = ((8, 8), (16, 16), (16, 8), (32, 16), (32, 32))


def load_cases():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b = line.split("|")
        f = a.split()
        rows.append(([float(x) for x in f[:6]], [int(x) for x in f[6:]], [int(x) for x in b.split()]))
    return rows


def test_hand_worked_cases():
    cases = load_cases()
    assert len(cases) >= 14
    for (u, v, sxx, sxy, syy, tau), (W, H, TW, TH), expect in cases:
        cnt, rect, cells = oracle.cull_f32([u], [v], [sxx], [sxy], [syy], [tau], [1], W, H, TW, TH)
        assert [cnt[0], *rect[0], cells[0]] == expect, (u, v, sxx, sxy, syy, tau, expect, cnt, rect, cells)
        keys, ids = oracle.emit_cull_keys([u], [v], [sxx], [sxy], [syy], [tau], [1], W, H, TW, TH, [1.0])
        assert len(keys) == cnt[0]


def random_gaussians(rng, n, W, H):
    """Screen-space Gaussians as the projection makes them: Sigma2 = R diag(s^2) R^T + 0.3 I
    with strong anisotropy and any angle, tau = 2 ln(255 o) capped at 2 ln 255."""
    u = rng.uniform(-15, W + 15, n)
    v = rng.uniform(-15, H + 15, n)
    s1 = np.exp(rng.normal(1.2, 0.9, n))
    s2 = s1 * np.exp(-rng.exponential(1.2, n))
    th = rng.uniform(0, np.pi, n)
    c, s = np.cos(th), np.sin(th)
    sxx = c * c * s1 ** 2 + s * s * s2 ** 2 + 0.3
    syy = s * s * s1 ** 2 + c * c * s2 ** 2 + 0.3
    sxy = c * s * (s1 ** 2 - s2 ** 2)
    o = rng.uniform(0.002, 0.995, n)
    tau = np.minimum(2 * np.log(255 * o), 2 * np.log(255.0))
    f = lambda a: a.astype(np.float32)
    return f(u), f(v), f(sxx), f(sxy), f(syy), f(tau)


def kept_tiles(u, v, sxx, sxy, syy, tau, W, H, TW, TH):
    n = len(u)
    keys, ids = oracle.emit_cull_keys(u, v, sxx, sxy, syy, tau, np.ones(n, np.uint8), W, H, TW, TH,
                                      np.zeros(n, np.float32))
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    kept = [set() for _ in range(n)]
    for t, i in zip(tiles, ids):
        kept[i].add(int(t))
    return kept


def conic64(sxx, sxy, syy):
    a, b, c = (np.float64(x) for x in (sxx, sxy, syy))
    det = a * c - b * b
    return c / det, -b / det, a / det


def test_conservative_against_brute_force():
    """Every pixel centre strictly inside the ellipse (FP64, 1e-5 margin for FP32 rounding)
    has its tile kept, for every tile shape."""
    rng = np.random.default_rng(11)
    W, H, n = 96, 64, 400
    g = random_gaussians(rng, n, W, H)
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    for TW, TH in TILES:
        kept = kept_tiles(*g, W, H, TW, TH)
        tile_of = (ys.astype(int) // TH) * ((W + TW - 1) // TW) + xs.astype(int) // TW
        for i in range(n):
            A, B, C = conic64(g[2][i], g[3][i], g[4][i])
            dx, dy = xs - np.float64(g[0][i]), ys - np.float64(g[1][i])
            inside = A * dx * dx + 2 * B * dx * dy + C * dy * dy <= np.float64(g[5][i]) * (1 - 1e-5)
            need = set(np.unique(tile_of[inside]).tolist())
            assert need <= kept[i], (TW, TH, i, sorted(need - kept[i]))


def near_singular(sxx, sxy, syy):
    """The rule's FP32 test a c > 64 det (such footprints keep their whole extent box)."""
    ac = (sxx * syy).astype(np.float32)
    det = (ac - (sxy * sxy).astype(np.float32)).astype(np.float32)
    return ac > np.float32(64) * det


def test_tight_against_brute_force():
    """Every kept tile of a well-conditioned footprint has a pixel column (inside the extent
    box) whose centre line reaches the ellipse within the tile row's band (FP64 minimum of
    the quadratic form over the band, 1e-4 relative margin)."""
    rng = np.random.default_rng(12)
    W, H, n = 96, 64, 400
    g = random_gaussians(rng, n, W, H)
    for TW, TH in TILES:
        kept = kept_tiles(*g, W, H, TW, TH)
        _, rect, _ = oracle.cull_f32(*g, np.ones(n, np.uint8), W, H, TW, TH)
        tiles_x = (W + TW - 1) // TW
        n_culled = 0
        skip = near_singular(g[2], g[3], g[4])
        assert 0 < skip.sum() < n // 4
        for i in range(n):
            if not kept[i] or skip[i]:
                continue
            u, v, tau = (np.float64(g[k][i]) for k in (0, 1, 5))
            A, B, C = conic64(g[2][i], g[3][i], g[4][i])
            ex, ey = np.sqrt(tau * np.float64(g[2][i])), np.sqrt(tau * np.float64(g[4][i]))
            px0, px1 = max(np.ceil(u - ex - 0.5), 0), min(np.floor(u + ex - 0.5), W - 1)
            py0, py1 = max(np.ceil(v - ey - 0.5), 0), min(np.floor(v + ey - 0.5), H - 1)
            n_culled += (rect[i, 2] - rect[i, 0] + 1) * (rect[i, 3] - rect[i, 1] + 1) - len(kept[i])
            for t in kept[i]:
                ty, tx = divmod(t, tiles_x)
                cols = np.arange(max(tx * TW, px0), min(tx * TW + TW - 1, px1) + 1) + 0.5 - u
                d0 = max(ty * TH, py0) + 0.5 - v
                d1 = min(ty * TH + TH - 1, py1) + 0.5 - v
                dy = np.clip(-B * cols / C, d0, d1)  # minimiser over the band for each column
                q = A * cols * cols + 2 * B * cols * dy + C * dy * dy
                assert len(cols) and q.min() <= tau * (1 + 1e-4) + 1e-9, (TW, TH, i, t, q.min(), tau)
        assert n_culled > 0  # the random set exercises the cull


def test_near_singular_keeps_box_and_cull_never_adds():
    rng = np.random.default_rng(13)
    W, H, n = 128, 96, 300
    u, v, sxx, sxy, syy, tau = random_gaussians(rng, n, W, H)
    cnt, rect, cells = oracle.cull_f32(u, v, sxx, sxy, syy, tau, np.ones(n, np.uint8), W, H, 16, 16)
    assert np.all(cnt <= cells) and np.all(cells >= 0)
    ns = near_singular(sxx, sxy, syy)
    assert np.array_equal(cnt[ns], cells[ns])
    # made near-singular: sxy^2 close to sxx syy
    sxy_s = (np.sign(sxy) * np.sqrt(sxx.astype(np.float64) * syy) * (1 - 1e-4)).astype(np.float32)
    assert near_singular(sxx, sxy_s, syy).all()
    c2, _, cells2 = oracle.cull_f32(u, v, sxx, sxy_s, syy, tau, np.ones(n, np.uint8), W, H, 16, 16)
    assert np.array_equal(c2, cells2)


def test_emitted_keys_sorted_stably():
    """Keys sorted by (tile, depth bits), equal depths in emission order: numpy's stable
    sort equals Python's sort of (key, emit position); tiles are kept tiles only."""
    rng = np.random.default_rng(14)
    W, H, n = 80, 48, 300
    g = random_gaussians(rng, n, W, H)
    depth = rng.choice(np.array([2.0, 3.5, 7.25], np.float32), n)
    order = rng.permutation(n)
    keys, vals = oracle.emit_cull_keys(*g, np.ones(n, np.uint8), W, H, 16, 16, depth, order=order)
    cnt, _, _ = oracle.cull_f32(*g, np.ones(n, np.uint8), W, H, 16, 16)
    assert len(keys) == cnt.sum()
    # emission follows `order`
    first = {}
    for pos, i in enumerate(vals):
        first.setdefault(int(i), pos)
    seen = [int(i) for i in order if cnt[i] > 0]
    assert sorted(first, key=first.get) == seen
    sk, sv = oracle.sorted_keys(keys, vals)
    ref = sorted(range(len(keys)), key=lambda k: (int(keys[k]), k))
    assert np.array_equal(sv, vals[ref]) and np.array_equal(sk, keys[ref])
