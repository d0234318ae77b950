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
