"""The tile cover never drops a contributing (pixel, Gaussian) pair (GPU).

Eq. 2/3 composite, at every pixel, every Gaussian that passes the per-pixel
3-sigma cutoff and the 1/255 skip. Which Gaussians the blend evaluates at a
pixel is decided earlier, by the projection's FP32 tile cover (q_cover and a
box minimum of the quadratic form) and the emission. The bit-exact binning
tests compare those lists with the integer referee, which repeats the same
FP32 cover decisions from the GPU's own q_cover, so they pin the bookkeeping
(keys, order, ranges) but not the decision. These tests pin the decision
independently: from the FP64 oracle's own projection every contributing pixel
is enumerated by brute force (tests/cover_check.py, itself pinned on the CPU
against planted mistakes) and the GPU's sorted list of that pixel's tile must
hold the Gaussian. They also check every visible record's q_cover against the
FP64 bound min(9, 2 ln(255 o)).
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_03737_gb300 import scenes
from tests.cover_check import check_cover, listed_pairs, q_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2507_03737_gb300.autograd import Renderer
    r = Renderer(0)
    yield r
    r.close()


def _ragged():
    """Config-1 Gaussians seen by five uneven, shifted cameras (one of 1 x 1 pixels)."""
    sc = scenes.config_scene(1, n_override=3000)
    base = sc.cameras[0]
    rng = np.random.default_rng(2)
    cams = [base]
    for (w, h) in [(37, 53), (161, 7), (1, 1), (64, 48)]:
        T = scenes.look_at_pose(rng.uniform(-0.5, 0.5, 3), yaw=rng.uniform(-0.1, 0.1))
        cams.append(scenes.camera(w, h, 150.0, 150.0, w / 2 + rng.uniform(-9, 9), h / 2 + rng.uniform(-9, 9), T))
    sc.cameras = cams
    return sc


def _case(name):
    if name == "config1":
        return scenes.config_scene(1)
    if name == "ragged":
        return _ragged()
    if name == "config3_50k_2views":
        sc = scenes.config_scene(3, n_override=50_000)
        sc.cameras = sc.cameras[:2]
        return sc
    if name == "config5_20k_2views":
        # large, elongated Gaussians (log-scale N(log 0.1, 0.8^2)), SH 3, both view sizes
        sc = scenes.config_scene(5, n_override=20_000)
        sc.cameras = sc.cameras[:2]
        return sc
    raise ValueError(name)


CASES = [("config1", (16, 16)), ("config1", (8, 8)), ("config1", (32, 8)), ("ragged", (16, 16)),
         ("ragged", (8, 8)), ("config3_50k_2views", (16, 16)), ("config3_50k_2views", (8, 8)),
         ("config5_20k_2views", (16, 16))]


@pytest.mark.parametrize("name,tile", CASES, ids=[f"{n}-{t[0]}x{t[1]}" for n, t in CASES])
def test_cover_lists_every_contributing_pair(R, name, tile):
    from paper_2507_03737_gb300 import binding as B
    sc = _case(name)
    R.render_np(sc, options=B.s3gs_options_default(tile_w=tile[0], tile_h=tile[1], full_lists=1))
    keys, vals, _ = B.s3gs_debug_binning(R.ctx, R.state)
    res = check_cover(sc, sc.cameras, listed_pairs(keys, vals), tile[0], tile[1])
    print(f"COVER {name} {tile[0]}x{tile[1]}: {res}")
    assert res["records"] > 0.3 * min(sc.n, 20_000), res
    assert res["missing"] == 0, res
    # the band of FP32-sensitive pairs is a small part of what is checked
    assert res["band_pairs"] <= 0.002 * res["pixel_pairs"] + 10, res


@pytest.mark.parametrize("name", ["config1", "ragged", "config3_50k_2views", "config5_20k_2views"])
def test_q_cover_not_below_the_fp64_bound(R, name):
    """q_cover >= min(9, 2 ln(255 o)) for every record, with the FP32 widening the
    projection claims (relative 1e-5 of it must be visible) and an absolute 1e-5 for
    the FP32 rounding of log2(opacity), which matters only where o is near 1/255."""
    from paper_2507_03737_gb300 import binding as B
    sc = _case(name)
    V, n = len(sc.cameras), sc.n
    R.render_np(sc)
    qc = B.s3gs_debug_cover(R.ctx, R.state, n * V).astype(np.float64).reshape(V, n)
    rec = B.s3gs_debug_records(R.ctx, R.state, n * V)
    vis = (rec["extent"][:, 0] > 0).reshape(V, n)
    checked = 0
    for k, cam in enumerate(sc.cameras):
        p = O.project(sc, cam)
        both = vis[k] & (p["valid"] > 0)
        qb = q_bound(p["opacity"][both])
        bad = qc[k][both] < qb * (1 + 1e-5) - 1e-5
        assert not bad.any(), (k, qc[k][both][bad][:5], qb[bad][:5])
        checked += int(both.sum())
    print(f"QCOVER {name}: {checked} records")
    assert checked > 0.3 * min(n, 20_000)
