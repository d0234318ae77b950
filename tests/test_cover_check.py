"""Pins of the brute-force cover check (tests/cover_check.py) on the CPU.

The GPU test of the tile cover asks whether the library's sorted tile lists hold
every (pixel, Gaussian) pair that contributes to Eq. 2/3 by the FP64 oracle's
projection. Here the check itself is shown to tell a correct cover from
plausible mistakes: lists built by the integer referee with the full bound
q_b = min(9, 2 ln(255 o)) (slightly widened, as a cover must be) pass, and
lists built with q_cover tightened by 1 % or by 0.3 %, with the 1/255 skip
bound taken with a base-10 logarithm, with the conic's off-diagonal sign
flipped, or with the bounding rectangle one pixel short, fail. The mistakes are planted in the
referee's inputs, on the CPU; no kernel is changed.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2507_03737_gb300 import scenes
from tests.cover_check import check_cover, listed_pairs, q_bound


def _referee_inputs(sc, cams, qc_scale=1.0, qc_fn=None, b_sign=1.0, ext_delta=0):
    """FP32 records of the oracle's projection, as the renderer's cover consumes them."""
    n = sc.n
    V = len(cams)
    u = np.zeros(V * n, np.float32); v = np.zeros_like(u); z = np.zeros_like(u)
    rx = np.zeros(V * n, np.int32); ry = np.zeros_like(rx)
    conic = np.zeros((V * n, 3), np.float32); qc = np.zeros(V * n, np.float32)
    for k, cam in enumerate(cams):
        p = O.project(sc, cam)
        ok = p["valid"] > 0
        A, B, C = p["A"], p["B"], p["C"]
        det = A * C - B * B
        with np.errstate(divide="ignore", invalid="ignore"):
            cxx, cyy = C / det, A / det
            tr, dd = A + C, np.sqrt(np.maximum((A - C) ** 2 + 4 * B * B, 0))
            kappa = (tr + dd) / np.maximum(tr - dd, 1e-300)
            ex = np.ceil(3.0 * np.sqrt(cxx) * (1 + 1e-5 + 4e-7 * kappa) + 0.01) + ext_delta
            ey = np.ceil(3.0 * np.sqrt(cyy) * (1 + 1e-5 + 4e-7 * kappa) + 0.01) + ext_delta
        qb = q_bound(p["opacity"]) if qc_fn is None else qc_fn(p["opacity"])
        sl = slice(k * n, (k + 1) * n)
        ok = ok & (qb > 0)
        u[sl] = np.where(ok, p["u"], 0); v[sl] = np.where(ok, p["v"], 0); z[sl] = np.where(ok, p["depth"], 1)
        rx[sl] = np.where(ok, ex, 0); ry[sl] = np.where(ok, ey, 0)
        conic[sl] = np.stack([np.where(ok, A, 1), np.where(ok, b_sign * B, 0), np.where(ok, C, 1)], 1)
        qc[sl] = np.where(ok, qb * (1 + 2e-5 + 8e-7 * kappa) * qc_scale, 0)
    return [(c["width"], c["height"]) for c in cams], u, v, rx, ry, z, conic, qc


def _scene():
    sc = scenes.config_scene(1, n_override=1500)
    rng = np.random.default_rng(5)
    # elongated, rotated Gaussians so that the off-diagonal of the conic matters
    sc.log_scales[:, 0] += np.float32(1.0)
    sc.log_scales[:, 1] -= np.float32(0.5)
    cams = [sc.cameras[0], scenes.camera(61, 45, 80.0, 80.0, 30.0 + rng.uniform(-3, 3), 22.0,
                                         scenes.look_at_pose(np.array([0.3, -0.2, 0.5]), yaw=0.05))]
    sc.cameras = cams
    return sc


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_correct_cover_passes(tile):
    sc = _scene()
    wh, u, v, rx, ry, z, conic, qc = _referee_inputs(sc, sc.cameras)
    keys, vals, _ = O.bin_referee(wh, tile[0], tile[1], u, v, rx, ry, z, conic=conic, q_cover=qc)
    res = check_cover(sc, sc.cameras, listed_pairs(keys, vals), tile[0], tile[1])
    assert res["required"] > 2000 and res["pixel_pairs"] > 50000, res
    assert res["missing"] == 0, res
    assert res["band_pairs"] < 0.01 * res["pixel_pairs"], res


@pytest.mark.parametrize("mistake", ["tight1pct", "tight03pct", "log10_skip", "b_sign", "rect_short"])
def test_planted_cover_mistakes_are_caught(mistake):
    sc = _scene()
    kw = dict(tight1pct=dict(qc_scale=0.99), tight03pct=dict(qc_scale=0.997),
              log10_skip=dict(qc_fn=lambda o: np.minimum(9.0, 2.0 * np.log10(np.maximum(255.0 * o, 1e-30)))),
              b_sign=dict(b_sign=-1.0),
              rect_short=dict(ext_delta=-1))[mistake]
    wh, u, v, rx, ry, z, conic, qc = _referee_inputs(sc, sc.cameras, **kw)
    keys, vals, _ = O.bin_referee(wh, 16, 16, u, v, rx, ry, z, conic=conic, q_cover=qc)
    res = check_cover(sc, sc.cameras, listed_pairs(keys, vals), 16, 16)
    assert res["missing"] > 0, res


def test_q_bound_closed_form():
    # 9 for o >= e^4.5 / 255 (3-sigma cutoff binds), 2 ln(255 o) below (1/255 skip binds)
    o = np.array([1.0, 0.5, math.exp(4.5) / 255.0, 0.1, 1.0 / 255.0, 0.5 / 255.0])
    qb = q_bound(o)
    assert qb[0] == 9.0 and qb[1] == 9.0
    assert abs(qb[2] - 9.0) < 1e-12
    assert abs(qb[3] - 2 * math.log(25.5)) < 1e-12
    assert qb[4] == 0.0 and qb[5] < 0
    # at q = q_b the pair's alpha is exactly 1/255 (or q = 9)
    a = o[3] * math.exp(-0.5 * qb[3])
    assert abs(a - 1.0 / 255.0) < 1e-15
