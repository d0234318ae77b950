"""Parity at the full workload sizes, in the launch configuration bench.py times.

The GPU renders every view of a workload in one batched call with the default
options; the FP64 oracle renders small crop windows of those views (a crop is
the same camera with a shifted principal point, so its pixels equal that
window of the full render). Gradients are checked with upstream gradients that
are nonzero only inside the crops (and only on pixels whose FP64 decisions are
clear of every threshold), so the oracle's crop backward is the exact
reference for the full-size GPU backward.

At these densities a pixel evaluates hundreds of Gaussians, and each decision
(3-sigma cutoff, 1/255 skip, 0.99 clamp, 1e-4 stop, depth order) has a small
chance of lying within the 1e-5 relative margin at which FP32 and FP64 may
decide differently; such pixels are excluded and counted (each test bounds the
count by what was measured plus slack), and every test still compares several
hundred pixels.
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_03737_gb300 import scenes
from tests.gpu_helpers import TOL_GRAD, compare_forward, pixel_mask, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2507_03737_gb300.autograd import Renderer
    r = Renderer(0)
    yield r
    r.close()


def _crops(cameras, per_view, w, h, seed):
    """Seeded crop windows: (view, x0, y0, crop camera)."""
    rng = np.random.default_rng(seed)
    out = []
    for v, cam in enumerate(cameras):
        for _ in range(per_view):
            x0 = int(rng.integers(0, cam["width"] - w + 1))
            y0 = int(rng.integers(0, cam["height"] - h + 1))
            crop = dict(cam, width=w, height=h, cx=cam["cx"] - x0, cy=cam["cy"] - y0)
            out.append((v, x0, y0, crop))
    return out


def _window(full, cameras, key, ch, v, x0, y0, w, h):
    off = sum(c["width"] * c["height"] for c in cameras[:v])
    cam = cameras[v]
    plane = full[key][ch * off: ch * (off + cam["width"] * cam["height"])].reshape(ch, cam["height"], cam["width"])
    return plane[:, y0:y0 + h, x0:x0 + w].reshape(-1)


def _forward_check(R, sc, crops, w, h, options=None, max_excluded=0.01):
    full = R.render_np(sc, options=options)
    crop_cams = [c for (_, _, _, c) in crops]
    ref = O.render_fwd(sc, cameras=crop_cams)
    gpu = {k: [] for k in ("rgb", "depth", "pointmap", "alpha")}
    for (v, x0, y0, _) in crops:
        for k, ch in (("rgb", 3), ("depth", 1), ("pointmap", 3), ("alpha", 1)):
            gpu[k].append(_window(full, sc.cameras, k, ch, v, x0, y0, w, h))
    gpu = {k: np.concatenate(x) for k, x in gpu.items()}
    res = compare_forward(gpu, ref, crop_cams, max_excluded=max_excluded)
    assert res["pixels"] - res["excluded"] >= 300, res
    return ref, res


def _sparse_upstream(sc, crops, w, h, ref, seed):
    """Full-size upstream gradients, nonzero only on clear pixels of the crops;
    returns them and the matching per-crop arrays for the oracle."""
    rng = np.random.default_rng(seed)
    P = sum(c["width"] * c["height"] for c in sc.cameras)
    full = dict(d_rgb=np.zeros(3 * P), d_depth=np.zeros(P), d_pointmap=np.zeros(3 * P), d_alpha=np.zeros(P))
    per = dict(d_rgb=[], d_depth=[], d_pointmap=[], d_alpha=[])
    mask = pixel_mask(ref)
    for ci, (v, x0, y0, crop) in enumerate(crops):
        m = mask[ci * w * h:(ci + 1) * w * h].reshape(h, w)
        cam = sc.cameras[v]
        off = sum(c["width"] * c["height"] for c in sc.cameras[:v])
        HW = cam["width"] * cam["height"]
        for key, ch in (("d_rgb", 3), ("d_depth", 1), ("d_pointmap", 3), ("d_alpha", 1)):
            vals = rng.standard_normal((ch, h, w)) * m[None]
            per[key].append(vals.reshape(-1))
            plane = full[key][ch * off: ch * (off + HW)].reshape(ch, cam["height"], cam["width"])
            plane[:, y0:y0 + h, x0:x0 + w] += vals
    return full, {k: np.concatenate(x) for k, x in per.items()}


def _twist_by_view(twist_crops, crops, n_views):
    out = np.zeros((n_views, 6))
    for (v, _, _, _), t in zip(crops, twist_crops):
        out[v] += t
    return out


# the library default, and the schedule the autotuner picks for config 3 (a persistent
# heaviest-first grid of 12 CTAs per SM, 4 pixels per backward thread, batches of 128)
CONFIG3_SCHEDULES = [None, dict(blocks_per_sm=12, pixels_per_thread=2, bwd_pixels_per_thread=4, batch=128)]


@pytest.mark.parametrize("schedule", CONFIG3_SCHEDULES, ids=["default", "autotuned"])
def test_config3_full_size_window(R, schedule):
    """1M Gaussians, 12 x 1241x376, batched: forward windows and sparse-gradient backward."""
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.config_scene(3)
    w, h = 32, 24
    crops = _crops(sc.cameras, 1, w, h, seed=31)
    options = None if schedule is None else B.s3gs_options_default(**schedule)
    ref, res = _forward_check(R, sc, crops, w, h, options=options, max_excluded=0.005)
    assert res["pixels"] == 12 * w * h
    full_ups, crop_ups = _sparse_upstream(sc, crops, w, h, ref, seed=32)
    g = R.backward_np(full_ups, len(sc.cameras))
    gref = O.render_bwd(sc, cameras=[c for (_, _, _, c) in crops], **crop_ups)
    for k in ("means", "log_scales", "quats", "opacity_logits", "colors"):
        assert rel_l2(g[k], gref[k]) <= TOL_GRAD, k
    tw = _twist_by_view(gref["twist"], crops, len(sc.cameras))
    assert rel_l2(g["twist"], tw) <= TOL_GRAD


def test_config2_full_size_sh3(R):
    """500k Gaussians with SH degree 3 on one 1241x376 driving frame."""
    sc = scenes.config_scene(2)
    w, h = 16, 12
    crops = _crops(sc.cameras, 4, w, h, seed=21)
    ref, _ = _forward_check(R, sc, crops, w, h)
    full_ups, crop_ups = _sparse_upstream(sc, crops, w, h, ref, seed=22)
    g = R.backward_np(full_ups, 1)
    gref = O.render_bwd(sc, cameras=[c for (_, _, _, c) in crops], **crop_ups)
    for k in ("means", "log_scales", "quats", "opacity_logits", "colors", "twist"):
        ref_k = gref[k] if k != "twist" else _twist_by_view(gref[k], crops, 1)
        assert rel_l2(g[k], ref_k) <= TOL_GRAD, k


def test_config4_pose_only_uneven(R):
    """2M Gaussians, 16 views of three resolutions, pose-only backward (tracking)."""
    import torch
    sc = scenes.config_scene(4)
    w, h = 12, 8
    crops = _crops(sc.cameras, 1, w, h, seed=41)[::2]  # every other view
    ref, _ = _forward_check(R, sc, crops, w, h)
    full_ups, crop_ups = _sparse_upstream(sc, crops, w, h, ref, seed=42)
    g = R.backward_np(full_ups, len(sc.cameras), want=("twist",))
    assert set(g) == {"twist"}
    gref = O.render_bwd(sc, cameras=[c for (_, _, _, c) in crops], **crop_ups)
    tw = _twist_by_view(gref["twist"], crops, len(sc.cameras))
    assert rel_l2(g["twist"], tw) <= TOL_GRAD


def test_config5_crop_deterministic_vs_atomic(R):
    """5M Gaussians, SH degree 3, log-scales N(log 0.1, 0.8^2): deterministic and atomic
    gradients (recomputed blend state) against the oracle on a 64x48 crop of view 0."""
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.config_scene(5)
    cam = sc.cameras[0]
    crop = dict(cam, width=64, height=48, cx=cam["cx"] - 580, cy=cam["cy"] - 160)
    ref = O.render_fwd(sc, cameras=[crop])
    mask = pixel_mask(ref)
    rng = np.random.default_rng(51)
    P = 64 * 48
    ups = dict(d_rgb=rng.standard_normal(3 * P) * np.tile(mask, 3), d_depth=rng.standard_normal(P) * mask,
               d_pointmap=rng.standard_normal(3 * P) * np.tile(mask, 3), d_alpha=rng.standard_normal(P) * mask)
    gref = O.render_bwd(sc, cameras=[crop], **ups)
    grads = {}
    for det in (0, 1):
        opt = B.s3gs_options_default(deterministic=det, recompute=1)
        gpu = R.render_np(sc, cameras=[crop], options=opt)
        compare_forward(gpu, ref, [crop], max_excluded=0.005)
        grads[det] = R.backward_np(ups, 1)
        for k in ("means", "log_scales", "quats", "opacity_logits", "colors", "twist"):
            assert rel_l2(grads[det][k], gref[k]) <= TOL_GRAD, (det, k)
    R.render_np(sc, cameras=[crop], options=B.s3gs_options_default(deterministic=1, recompute=1))
    again = R.backward_np(ups, 1)
    for k in again:
        np.testing.assert_array_equal(again[k], grads[1][k])


def _pixel_changed(a, b, cameras):
    """Per pixel: does any output differ by more than the parity tolerances?"""
    P = sum(c["width"] * c["height"] for c in cameras)
    ch = np.zeros(P, bool)
    for k, c in (("rgb", 3), ("pointmap", 3), ("depth", 1), ("alpha", 1)):
        x = a[k].astype(np.float64).reshape(-1)
        y = b[k].astype(np.float64).reshape(-1)
        tol = 1e-4 if k in ("rgb", "alpha") else 1e-4 * np.abs(y) + 1e-6
        d = (np.abs(x - y) > tol)
        if c == 3:
            off, parts = 0, []
            for cam in cameras:
                hw = cam["width"] * cam["height"]
                parts.append(d[3 * off: 3 * (off + hw)].reshape(3, hw).any(0))
                off += hw
            d = np.concatenate(parts)
        ch |= d
    return ch


@pytest.mark.parametrize("cid", [1, 3])
def test_guard_cone_effect_on_workloads(R, cid):
    """What the guard cone (default) changes in the renders of configs 1 and 3, against
    the plain projection without it: the records it culls and the fraction of pixels
    with any output changed beyond the parity tolerances (printed for the record).
    The cone only ever removes records, and every record it removes has its mean
    outside the cone, |x/z| > 1.5 or |y/z| > 1.5 (read from the record's own centre,
    x/z = (u - c_x) / f_x)."""
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.config_scene(cid)
    V, n = len(sc.cameras), sc.n
    on = R.render_np(sc)
    vis_on = B.s3gs_debug_records(R.ctx, R.state, V * n)["extent"][:, 0] > 0
    off = R.render_np(sc, options=B.s3gs_options_default(guard_slope=-1.0))
    rec_off = B.s3gs_debug_records(R.ctx, R.state, V * n)
    vis_off = rec_off["extent"][:, 0] > 0
    assert not (vis_on & ~vis_off).any()
    only = np.nonzero(vis_off & ~vis_on)[0]
    view = only // n
    fx = np.array([c["fx"] for c in sc.cameras])[view]
    fy = np.array([c["fy"] for c in sc.cameras])[view]
    cx = np.array([c["cx"] for c in sc.cameras])[view]
    cy = np.array([c["cy"] for c in sc.cameras])[view]
    sx = np.abs(rec_off["xy"][only, 0] - cx) / fx
    sy = np.abs(rec_off["xy"][only, 1] - cy) / fy
    assert np.all(np.maximum(sx, sy) > 1.5 * (1 - 1e-4))
    changed = _pixel_changed(on, off, sc.cameras)
    z = rec_off["rgb_depth"][only, 3]
    print(f"GUARD config {cid}: records culled by the cone {only.size} of {int(vis_off.sum())} "
          f"(z {float(z.min()) if only.size else 0:.3f}-{float(z.max()) if only.size else 0:.3f} m); "
          f"pixels changed {int(changed.sum())} of {changed.size} ({changed.mean():.4%})")
    if cid == 1:
        assert only.size == 0 and not changed.any()


def test_config3_binning_bit_exact_at_full_size(R):
    """The whole config-3 duplicate list (every tile of 12 x 1241x376) equals the
    integer referee's stable sort of the same records' cover, bit for bit."""
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.config_scene(3)
    R.render_np(sc, options=B.s3gs_options_default(full_lists=1))
    V = len(sc.cameras)
    rec = B.s3gs_debug_records(R.ctx, R.state, V * sc.n)
    qc = B.s3gs_debug_cover(R.ctx, R.state, V * sc.n)
    keys, vals, ranges = B.s3gs_debug_binning(R.ctx, R.state)
    wh = [(c["width"], c["height"]) for c in sc.cameras]
    rk, rv, rr = O.bin_referee(wh, 16, 16, rec["xy"][:, 0], rec["xy"][:, 1], rec["extent"][:, 0],
                               rec["extent"][:, 1], rec["rgb_depth"][:, 3], conic=rec["conic_opacity"][:, :3],
                               q_cover=qc)
    assert keys.size == rk.size > 10_000_000
    assert np.array_equal(keys, rk) and np.array_equal(vals, rv) and np.array_equal(ranges, rr)
