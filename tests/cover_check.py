"""Brute-force check that a tile list holds every contributing (pixel, Gaussian) pair.

A Gaussian contributes to a pixel's composite (Eq. 2, Eq. 3) when the pixel
passes its 3-sigma cutoff, q = d^T Sigma'^-1 d <= 9, and its alpha
o exp(-q / 2) is not skipped as below 1/255. Both are one bound on q:

    q <= q_b = min(9, 2 ln(255 o)).

The tile cover only has to list, for every such pair, the Gaussian in the
tile that holds the pixel. This module enumerates those pairs from the FP64
oracle's own projection (centre, conic, opacity: no value computed on the GPU
decides anything here), pixel by pixel over the ellipse's bounding box, and
reports which of them a given list of (global tile, Gaussian) pairs lacks.

A pair whose FP64 q lies within ``band`` of q_b is left out and counted: the
renderer computes the centre and the conic in FP32, which moves q by up to

    band = 2 sqrt(q_b lambda_max(Sigma'^-1)) delta + q_b (1e-5 + 2e-6 kappa) + 1e-5,

where delta bounds the FP32 error of the centre in pixels (a few roundings of
x = R m + t at the magnitude of the mean and the translation, scaled by f / z,
plus the rounding of u itself) and kappa is the condition number of Sigma'.
Records culled by the near plane or the guard cone within a relative 1e-4 of
the decision are left out as well.
"""
from __future__ import annotations

import numpy as np

EPS32 = 2.0 ** -24


def q_bound(opacity):
    """min(9, 2 ln(255 o)): the largest q at which a pair contributes."""
    o = np.asarray(opacity, np.float64)
    with np.errstate(divide="ignore"):
        return np.minimum(9.0, 2.0 * np.log(255.0 * o))


def _tiles_of_view(cam, tw, th):
    return (cam["width"] + tw - 1) // tw, (cam["height"] + th - 1) // th


def contributing_pairs(proj, cam, mean_norm, t_norm, tile_base, tw, th, guard=1.5, near_z=0.2,
                       chunk=4_000_000):
    """Enumerate the contributing (pixel, Gaussian) pairs of one view.

    proj: the oracle's per-Gaussian FP64 projection for this camera (``oracle.project``).
    mean_norm, t_norm: |mean| per Gaussian and |t| of the pose (FP32 error model).
    Returns (pairs, n_tested, n_band, n_records): pairs as uint64 (global tile << 32 | g),
    the number of enumerated pairs checked, the number left out in the band, and the
    number of records that have at least one contributing pixel.
    """
    W, H = int(cam["width"]), int(cam["height"])
    fx, fy, cx, cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    tiles_x, _ = _tiles_of_view(cam, tw, th)
    valid = proj["valid"] > 0
    u, v, z = proj["u"], proj["v"], proj["depth"]
    A, B, C = proj["A"], proj["B"], proj["C"]
    o = proj["opacity"]
    # near plane / guard cone: leave out records whose decision is within 1e-4
    sx = np.abs((u - cx) / fx)
    sy = np.abs((v - cy) / fy)
    cm = np.abs(z - near_z) / near_z
    if guard > 0:
        cm = np.minimum(cm, np.minimum(np.abs(sx - guard), np.abs(sy - guard)) / guard)
    qb = q_bound(o)
    keep = valid & (cm > 1e-4) & (qb > 0)
    g_idx = np.nonzero(keep)[0]
    if g_idx.size == 0:
        return np.zeros(0, np.uint64), 0, 0, 0
    u, v, z, A, B, C, qb = (x[g_idx] for x in (u, v, z, A, B, C, qb))
    det = A * C - B * B
    cov_xx, cov_yy = C / det, A / det  # Sigma' = inverse of the conic
    tr, dd = A + C, np.sqrt(np.maximum((A - C) ** 2 + 4 * B * B, 0.0))
    lam_max, lam_min = 0.5 * (tr + dd), 0.5 * (tr - dd)
    kappa = lam_max / np.maximum(lam_min, 1e-300)
    mag = mean_norm[g_idx] + t_norm
    slope = 1.0 + np.abs((u - cx) / fx) + np.abs((v - cy) / fy)
    delta = 2.0 * (3.0 * EPS32 * max(fx, fy) * mag * slope / z + 2.0 * EPS32 * (np.abs(u) + np.abs(v) + abs(cx) + abs(cy)))
    band = 2.0 * np.sqrt(qb * lam_max) * delta + qb * (1e-5 + 2e-6 * kappa) + 1e-5
    # pixel box of the ellipse q <= q_b (exact half-extents sqrt(q_b Sigma'_xx), sqrt(q_b Sigma'_yy))
    hx, hy = np.sqrt(qb * cov_xx), np.sqrt(qb * cov_yy)
    x0 = np.maximum(np.ceil(u - hx), 0).astype(np.int64)
    x1 = np.minimum(np.floor(u + hx), W - 1).astype(np.int64)
    y0 = np.maximum(np.ceil(v - hy), 0).astype(np.int64)
    y1 = np.minimum(np.floor(v + hy), H - 1).astype(np.int64)
    nx, ny = np.maximum(x1 - x0 + 1, 0), np.maximum(y1 - y0 + 1, 0)
    cnt = nx * ny
    out, n_tested, n_band = [], 0, 0
    contributing = np.zeros(g_idx.size, bool)
    start = 0
    csum = np.cumsum(cnt)
    while start < g_idx.size:
        # records [start, stop) with at most ``chunk`` pixels in total (at least one record)
        base = csum[start - 1] if start > 0 else 0
        stop = int(np.searchsorted(csum, base + chunk, side="right"))
        stop = max(stop, start + 1)
        sl = slice(start, stop)
        c = cnt[sl]
        tot = int(c.sum())
        if tot:
            rec = np.repeat(np.arange(start, stop), c)
            first = np.repeat(np.cumsum(c) - c, c)
            loc = np.arange(tot) - first
            px = x0[rec] + loc % nx[rec]
            py = y0[rec] + loc // nx[rec]
            dx, dy = px - u[rec], py - v[rec]
            q = A[rec] * dx * dx + 2.0 * B[rec] * dx * dy + C[rec] * dy * dy
            inside = q <= qb[rec]
            sure = q <= qb[rec] - band[rec]
            n_band += int((inside & ~sure).sum())
            n_tested += int(sure.sum())
            contributing[np.unique(rec[sure])] = True
            tile = tile_base + (py[sure] // th) * tiles_x + (px[sure] // tw)
            out.append((tile.astype(np.uint64) << np.uint64(32)) | g_idx[rec[sure]].astype(np.uint64))
        start = stop
    pairs = np.unique(np.concatenate(out)) if out else np.zeros(0, np.uint64)
    return pairs, n_tested, n_band, int(contributing.sum())


def check_cover(scene, cameras, listed, tw, th, guard=1.5, near_z=0.2):
    """Compare a tile list with the brute-force contributing set of every view.

    listed: uint64 array (global tile << 32 | Gaussian) of the pairs a tile list holds.
    Returns a dict with the number of (tile, Gaussian) pairs required, missing, the
    enumerated pixel pairs tested and left out in the band, and a few missing examples.
    """
    import oracle as O
    listed = np.unique(np.asarray(listed, np.uint64))
    mean_norm = np.linalg.norm(scene.means.astype(np.float64), axis=1)
    tile_base = 0
    req, miss, tested, band, recs = 0, 0, 0, 0, 0
    examples = []
    for vi, cam in enumerate(cameras):
        proj = O.project(scene, cam, near_z=near_z)
        T = np.asarray(cam["T_cw"], np.float64).reshape(3, 4)
        pairs, nt, nb, nr = contributing_pairs(proj, cam, mean_norm, float(np.linalg.norm(T[:, 3])),
                                               tile_base, tw, th, guard=guard, near_z=near_z)
        pos = np.searchsorted(listed, pairs)
        found = (pos < listed.size) & (listed[np.minimum(pos, max(listed.size - 1, 0))] == pairs)
        req += pairs.size
        miss += int((~found).sum())
        tested += nt
        band += nb
        recs += nr
        for p in pairs[~found][:5]:
            examples.append(dict(view=vi, tile=int(p >> np.uint64(32)), g=int(p & np.uint64(0xffffffff))))
        tx, ty = _tiles_of_view(cam, tw, th)
        tile_base += tx * ty
    return dict(required=req, missing=miss, pixel_pairs=tested, band_pairs=band, records=recs, examples=examples)


def listed_pairs(keys, values, ranges=None):
    """(global tile << 32 | Gaussian) of a sorted duplicate list whose keys carry the tile
    in their upper 32 bits and whose values are Gaussian indices."""
    keys = np.asarray(keys, np.uint64)
    tiles = keys >> np.uint64(32)
    return (tiles << np.uint64(32)) | np.asarray(values, np.uint64)
