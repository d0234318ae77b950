"""Pins of the integer binning referee (keys, stable sort, per-tile ranges).

The referee recomputes the tile binning from a record's FP32 centre and integer
half-extents. Here it is checked against a pixel-level brute force: a record
belongs to a tile iff at least one pixel of that tile lies in the record's
pixel rectangle.
"""
import math

import numpy as np

import oracle as O


def _records(rng, n_views, n, sizes):
    u = np.zeros(n_views * n, np.float32); v = np.zeros_like(u)
    rx = np.zeros(n_views * n, np.int32); ry = np.zeros_like(rx)
    z = np.zeros_like(u)
    for vv, (W, H) in enumerate(sizes):
        sl = slice(vv * n, (vv + 1) * n)
        u[sl] = rng.uniform(-10, W + 10, n).astype(np.float32)
        v[sl] = rng.uniform(-10, H + 10, n).astype(np.float32)
        rx[sl] = rng.integers(0, 9, n)
        ry[sl] = rng.integers(0, 9, n)
        # repeated depths so that stability (ties keep ascending index) is exercised
        z[sl] = rng.choice(np.float32([0.5, 1.0, 2.5, 7.0, 30.0]), n)
    return u, v, rx, ry, z


def test_referee_against_pixel_brute_force():
    rng = np.random.default_rng(7)
    sizes = [(37, 23), (16, 16), (50, 9)]
    n = 60
    tw, th = 16, 8
    u, v, rx, ry, z = _records(rng, len(sizes), n, sizes)
    keys, vals, ranges = O.bin_referee(sizes, tw, th, u, v, rx, ry, z)
    tile_base = [0]
    for W, H in sizes:
        tile_base.append(tile_base[-1] + math.ceil(W / tw) * math.ceil(H / th))
    expect = {t: [] for t in range(tile_base[-1])}
    for vv, (W, H) in enumerate(sizes):
        tx_n = math.ceil(W / tw)
        for g in range(n):
            r = vv * n + g
            if rx[r] <= 0 or ry[r] <= 0:
                continue
            xs = [i for i in range(W) if np.float32(u[r] - np.float32(rx[r])) <= i <= np.float32(u[r] + np.float32(rx[r]))]
            ys = [j for j in range(H) if np.float32(v[r] - np.float32(ry[r])) <= j <= np.float32(v[r] + np.float32(ry[r]))]
            tiles = sorted({tile_base[vv] + (j // th) * tx_n + (i // tw) for i in xs for j in ys})
            for t in tiles:
                expect[t].append((int(z[r].view(np.uint32)), g))
    assert len(keys) == sum(len(x) for x in expect.values())
    for t in range(tile_base[-1]):
        lo, hi = ranges[t], ranges[t + 1]
        got = [(int(k & 0xFFFFFFFF), int(vl)) for k, vl in zip(keys[lo:hi], vals[lo:hi])]
        assert all(int(k >> 32) == t for k in keys[lo:hi])
        assert got == sorted(expect[t]), t  # (depth bits, index): stable order of equal depths
    assert ranges[-1] == len(keys)
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)


def test_referee_empty_and_offscreen():
    u = np.float32([-50.0, 500.0]); v = np.float32([3.0, 3.0])
    rx = np.int32([3, 3]); ry = np.int32([3, 3]); z = np.float32([1.0, 1.0])
    keys, vals, ranges = O.bin_referee([(32, 16)], 16, 16, u, v, rx, ry, z)
    assert keys.size == 0 and np.all(ranges == 0)


def _golden_min(f, lo, hi, iters=200):
    """Minimum of a convex function on [lo, hi] by golden-section search."""
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(iters):
        if f(c) < f(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    return min(f(lo), f(hi), f(0.5 * (a + b)))


def test_ellipse_cover_against_numerical_box_minimum():
    """The ellipse test of the tile cover, checked per (record, tile) against an
    FP64 minimum of q over the tile's box of pixel centres found by golden-section
    search along the four edges (and 0 when the centre is inside). The cover must
    list every tile whose minimum is below q_cover (decisions within 1e-4 of it are
    not compared) and may list, besides, only tiles within its widening: a minimum
    at most 1 % (+ 0.01) above q_cover."""
    rng = np.random.default_rng(11)
    W, H, tw, th = 64, 48, 16, 8
    n = 300
    u = rng.uniform(-6, W + 6, n).astype(np.float32)
    v = rng.uniform(-6, H + 6, n).astype(np.float32)
    conic = np.zeros((n, 3), np.float32)
    rx = np.zeros(n, np.int32); ry = np.zeros(n, np.int32)
    for i in range(n):
        s1, s2 = rng.uniform(0.8, 9.0, 2)
        th_ = rng.uniform(0, math.pi)
        R = np.array([[math.cos(th_), -math.sin(th_)], [math.sin(th_), math.cos(th_)]])
        cov = R @ np.diag([s1 * s1, s2 * s2]) @ R.T
        con = np.linalg.inv(cov)
        conic[i] = [con[0, 0], con[0, 1], con[1, 1]]
        rx[i] = math.ceil(3.0 * math.sqrt(cov[0, 0]) + 0.01)
        ry[i] = math.ceil(3.0 * math.sqrt(cov[1, 1]) + 0.01)
    qc = rng.uniform(2.0, 9.0, n).astype(np.float32)
    z = np.float32(1.0) + np.arange(n, dtype=np.float32)
    keys, vals, _ = O.bin_referee([(W, H)], tw, th, u, v, rx, ry, z, conic=conic, q_cover=qc)
    listed = {(int(g), int(k >> np.uint64(32))) for k, g in zip(keys, vals)}
    rect_keys, rect_vals, _ = O.bin_referee([(W, H)], tw, th, u, v, rx, ry, z)
    compared = dropped = extra = 0
    for k, g in zip(rect_keys, rect_vals):
        g = int(g); t = int(k >> np.uint64(32))
        tx, ty = t % math.ceil(W / tw), t // math.ceil(W / tw)
        px0, px1 = tx * tw, min(tx * tw + tw - 1, W - 1)
        py0, py1 = ty * th, min(ty * th + th - 1, H - 1)
        A, B, C = (float(x) for x in conic[g])
        uu, vv = float(u[g]), float(v[g])
        q = lambda x, y: A * (x - uu) ** 2 + 2 * B * (x - uu) * (y - vv) + C * (y - vv) ** 2
        if px0 <= uu <= px1 and py0 <= vv <= py1:
            m = 0.0
        else:
            m = min(_golden_min(lambda y: q(px0, y), py0, py1), _golden_min(lambda y: q(px1, y), py0, py1),
                    _golden_min(lambda x: q(x, py0), px0, px1), _golden_min(lambda x: q(x, py1), px0, px1))
        q_c = float(qc[g])
        if abs(m - q_c) <= 1e-4 * q_c:
            continue
        compared += 1
        is_listed = (g, t) in listed
        if m <= q_c:
            assert is_listed, ("a tile the ellipse meets is missing", g, t, m, q_c)
        else:
            dropped += not is_listed
            extra += is_listed
            assert not is_listed or m <= 1.01 * q_c + 0.01, ("listed far outside the widening", g, t, m, q_c)
    assert compared > 500 and dropped > 50 and extra < 0.05 * compared
