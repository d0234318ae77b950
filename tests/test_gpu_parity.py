"""GPU path against the FP64 oracle through the C ABI (config 1 and variations).

Forward outputs element by element, binning bit-exactly against the integer
referee, gradients per tensor, plus the equivalences the design promises
(batched = per view, persistent = flat grid, recompute = stored state,
deterministic runs bitwise equal).
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_03737_gb300 import scenes
from tests.gpu_helpers import (compare_forward, compare_grads, expand3, pixel_mask, rel_l2,
                               upstream)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2507_03737_gb300.autograd import Renderer
    r = Renderer(0)
    yield r
    r.close()


def _opts(**kw):
    from paper_2507_03737_gb300 import binding as B
    return B.s3gs_options_default(**kw)


def test_projection_matches_oracle(R):
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.config_scene(1)
    R.render_np(sc)
    rec = B.s3gs_debug_records(R.ctx, R.state, sc.n)
    ref = O.project(sc, sc.cameras[0])
    vis = rec["extent"][:, 0] > 0
    assert vis.sum() > 0.5 * sc.n
    assert np.all(ref["valid"][vis] > 0)
    conic_norm = np.maximum(np.abs(ref["A"]), np.abs(ref["C"]))[vis]
    for k, col in (("u", rec["xy"][:, 0]), ("v", rec["xy"][:, 1]), ("A", rec["conic_opacity"][:, 0]),
                   ("B", rec["conic_opacity"][:, 1]), ("C", rec["conic_opacity"][:, 2]),
                   ("opacity", rec["conic_opacity"][:, 3]), ("depth", rec["rgb_depth"][:, 3]),
                   ("r", rec["rgb_depth"][:, 0])):
        a, b = col[vis].astype(np.float64), ref[k][vis]
        # conic entries relative to the conic's norm; pixel coordinates relative to |u| + 1 px
        scale = conic_norm if k in ("A", "B", "C") else np.abs(b) + (1.0 if k in ("u", "v") else 0.0)
        assert np.max(np.abs(a - b) / scale) < 2e-5, k


@pytest.mark.parametrize("tile", [(16, 16), (16, 8), (8, 8), (32, 8)])
def test_binning_bit_exact(R, tile):
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.tiny_scene(5, n=300, width=77, height=45, n_views=3, scale=0.2)
    sc.cameras[1] = dict(sc.cameras[1], width=33, height=70)
    sc.cameras[2] = dict(sc.cameras[2], width=16, height=16)
    opt = _opts(tile_w=tile[0], tile_h=tile[1], full_lists=1)
    R.render_np(sc, options=opt)
    rec = B.s3gs_debug_records(R.ctx, R.state, sc.n * 3)
    keys, vals, ranges = B.s3gs_debug_binning(R.ctx, R.state)
    wh = [(c["width"], c["height"]) for c in sc.cameras]
    qc = B.s3gs_debug_cover(R.ctx, R.state, sc.n * 3)
    rk, rv, rr = O.bin_referee(wh, tile[0], tile[1], rec["xy"][:, 0], rec["xy"][:, 1], rec["extent"][:, 0],
                               rec["extent"][:, 1], rec["rgb_depth"][:, 3], conic=rec["conic_opacity"][:, :3],
                               q_cover=qc)
    assert keys.size == rk.size > 0
    assert np.array_equal(keys, rk)
    assert np.array_equal(vals, rv)
    assert np.array_equal(ranges, rr)


# the library default, and the schedule bench.py times config 1 with (8x8 tiles,
# one pixel per thread, batches of 64)
CONFIG1_SCHEDULES = [None, dict(tile_w=8, tile_h=8, pixels_per_thread=1, bwd_pixels_per_thread=1, batch=64)]


@pytest.mark.parametrize("schedule", CONFIG1_SCHEDULES, ids=["default", "tuned"])
def test_forward_config1(R, schedule):
    sc = scenes.config_scene(1)
    gpu = R.render_np(sc, options=None if schedule is None else _opts(**schedule))
    ref = O.render_fwd(sc)
    res = compare_forward(gpu, ref, sc.cameras)
    assert res["excluded"] < 100


@pytest.mark.parametrize("guard", [1.5, -1.0], ids=["cone", "no_cone"])
@pytest.mark.parametrize("schedule", CONFIG1_SCHEDULES, ids=["default", "tuned"])
def test_backward_config1(R, schedule, guard):
    """Every gradient tensor and the twist, with the guard cone (default) and without it
    (the plain definition: config 1 has Gaussians out to |x/z| = 2, so the two differ)."""
    sc = scenes.config_scene(1)
    try:
        O.set_guard(guard)
        ref_f = O.render_fwd(sc)
        mask = pixel_mask(ref_f)
        ups = upstream(sc.cameras, 7, mask)
        kw = {} if schedule is None else dict(schedule)
        gpu_f = R.render_np(sc, options=_opts(guard_slope=guard, **kw))
        compare_forward(gpu_f, ref_f, sc.cameras)
        g = R.backward_np(ups, 1)
        gref = O.render_bwd(sc, **ups)
        compare_grads(g, gref)
    finally:
        O.set_guard(1.5)


@pytest.mark.parametrize("deg", [1, 3])
def test_sh_forward_backward(R, deg):
    sc = scenes.tiny_scene(61 + deg, n=40, width=40, height=30, sh_degree=deg, n_views=2, scale=0.2)
    ref_f = O.render_fwd(sc)
    gpu = R.render_np(sc)
    compare_forward(gpu, ref_f, sc.cameras)
    mask = pixel_mask(ref_f)
    ups = upstream(sc.cameras, 3, mask)
    g = R.backward_np(ups, 2)
    compare_grads(g, O.render_bwd(sc, **ups))


def test_multiview_uneven_ragged(R):
    """Uneven, non-multiple-of-tile resolutions and shifted principal points."""
    sc = scenes.config_scene(1, n_override=3000)
    base = sc.cameras[0]
    rng = np.random.default_rng(2)
    cams = [base]
    for (w, h) in [(37, 53), (161, 7), (1, 1), (64, 48)]:
        T = scenes.look_at_pose(rng.uniform(-0.5, 0.5, 3), yaw=rng.uniform(-0.1, 0.1))
        cams.append(scenes.camera(w, h, 150.0, 150.0, w / 2 + rng.uniform(-9, 9), h / 2 + rng.uniform(-9, 9), T))
    sc.cameras = cams
    ref_f = O.render_fwd(sc)
    for tile in [(16, 16), (8, 8), (32, 8)]:
        gpu = R.render_np(sc, options=_opts(tile_w=tile[0], tile_h=tile[1]))
        compare_forward(gpu, ref_f, cams)
    mask = pixel_mask(ref_f)
    ups = upstream(cams, 11, mask)
    g = R.backward_np(ups, len(cams))
    compare_grads(g, O.render_bwd(sc, **ups))


def test_crop_equals_window(R):
    """Shifted principal point: a crop equals the window of the full render (GPU vs GPU, bitwise
    up to the projection's rounding of u, v)."""
    sc = scenes.config_scene(1)
    full = R.render_np(sc)
    cam = sc.cameras[0]
    x0, y0, w, h = 37, 21, 64, 48
    crop = dict(cam, width=w, height=h, cx=cam["cx"] - x0, cy=cam["cy"] - y0)
    out = R.render_np(sc, cameras=[crop])
    ref = O.render_fwd(sc, cameras=[crop])
    compare_forward(out, ref, [crop])
    a = full["rgb"].reshape(3, 120, 160)[:, y0:y0 + h, x0:x0 + w]
    assert np.abs(out["rgb"].reshape(3, h, w) - a).max() < 1e-4


def test_batched_equals_per_view(R):
    import torch
    sc = scenes.tiny_scene(8, n=400, width=64, height=40, n_views=4, scale=0.15)
    full = R.render_np(sc)
    ups = upstream(sc.cameras, 4)
    g_all = R.backward_np(ups, 4)
    off = 0
    acc = None
    for v, cam in enumerate(sc.cameras):
        hw = cam["width"] * cam["height"]
        one = R.render_np(sc, cameras=[cam])
        for k, ch in (("rgb", 3), ("depth", 1), ("pointmap", 3), ("alpha", 1)):
            np.testing.assert_array_equal(one[k], full[k][ch * off: ch * (off + hw)])
        sub = {k: (u[3 * off: 3 * (off + hw)] if u.size == 3 * sum(c["width"] * c["height"] for c in sc.cameras)
                   else u[off: off + hw]) for k, u in ups.items()}
        g = R.backward_np(sub, 1)
        np.testing.assert_allclose(g["twist"][0], g_all["twist"][v], rtol=1e-4, atol=1e-4)
        acc = g if acc is None else {k: acc[k] + g[k] for k in acc if k != "twist"}
        off += hw
    for k in ("means", "log_scales", "quats", "opacity_logits", "colors"):
        assert rel_l2(g_all[k], acc[k]) < 1e-5, k


def test_persistent_and_recompute_and_det(R):
    """Every schedule against the oracle, and against the default schedule (outputs
    bitwise, gradients to 1e-5; deterministic mode bitwise)."""
    sc = scenes.tiny_scene(9, n=600, width=80, height=60, n_views=2, scale=0.15)
    ref = O.render_fwd(sc)
    ups = upstream(sc.cameras, 5, pixel_mask(ref))
    gref = O.render_bwd(sc, **ups)
    base = R.render_np(sc)
    # a dense scene (600 Gaussians over 80 x 60 pixels): 26 of 9,600 pixels lie in the band
    compare_forward(base, ref, sc.cameras, name="schedules default", max_excluded=0.004)
    g0 = R.backward_np(ups, 2)
    compare_grads(g0, gref)
    outs = {}
    for name, kw in (("persistent", dict(blocks_per_sm=2)), ("recompute", dict(recompute=1)),
                     ("ppt1", dict(pixels_per_thread=1, bwd_pixels_per_thread=1)),
                     ("ppt4_recompute", dict(pixels_per_thread=4, bwd_pixels_per_thread=2, recompute=1)),
                     ("det", dict(deterministic=1)), ("det_recompute", dict(deterministic=1, recompute=1)),
                     ("det_persistent", dict(deterministic=1, blocks_per_sm=3, batch=64)),
                     ("persistent16_ppt4", dict(blocks_per_sm=16, bwd_pixels_per_thread=4, batch=64))):
        out = R.render_np(sc, options=_opts(**kw))
        for k in base:
            np.testing.assert_array_equal(out[k], base[k], err_msg=f"{name} {k}")
        outs[name] = R.backward_np(ups, 2)
        compare_grads(outs[name], gref)
        for k in g0:
            assert rel_l2(outs[name][k], g0[k]) < 1e-5, (name, k)
    for k in g0:  # deterministic mode is bitwise reproducible, whatever the schedule
        np.testing.assert_array_equal(outs["det"][k], outs["det_recompute"][k])
        np.testing.assert_array_equal(outs["det"][k], outs["det_persistent"][k])
    R.render_np(sc, options=_opts(deterministic=1))
    again = R.backward_np(ups, 2)
    for k in g0:
        np.testing.assert_array_equal(again[k], outs["det"][k])


def test_batch_size_and_tile_do_not_change_forward(R):
    """Each tile shape, batch size and pixels-per-thread setting: the forward bitwise equal
    to the default's, which matches the oracle, and the gradients against the oracle."""
    sc = scenes.config_scene(1)
    ref = O.render_fwd(sc)
    ups = upstream(sc.cameras, 8, pixel_mask(ref))
    gref = O.render_bwd(sc, **ups)
    base = R.render_np(sc)
    compare_forward(base, ref, sc.cameras, name="tiles default")
    for kw in (dict(batch=32), dict(batch=1024), dict(tile_w=8, tile_h=8, batch=17, bwd_pixels_per_thread=2),
               dict(tile_w=32, tile_h=8),
               dict(pixels_per_thread=1), dict(pixels_per_thread=4, batch=100),
               dict(tile_w=16, tile_h=8, pixels_per_thread=4),
               dict(tile_w=8, tile_h=8, pixels_per_thread=1, bwd_pixels_per_thread=1)):
        out = R.render_np(sc, options=_opts(**kw))
        for k in base:
            np.testing.assert_array_equal(out[k], base[k], err_msg=str(kw))
        compare_grads(R.backward_np(ups, 1), gref)


def test_background_colour(R):
    sc = scenes.tiny_scene(10, n=30, width=30, height=20, scale=0.2)
    bg = (0.2, 0.5, 0.9)
    gpu = R.render_np(sc, options=_opts(bg=bg))
    ref = O.render_fwd(sc, bg=bg)
    compare_forward(gpu, ref, sc.cameras)
    mask = pixel_mask(ref)
    ups = upstream(sc.cameras, 2, mask)
    compare_grads(R.backward_np(ups, 1), O.render_bwd(sc, bg=bg, **ups))


def test_heavy_tile_sort_path(R):
    """Tiles with more than 4096 duplicates take the global-memory sort path."""
    from paper_2507_03737_gb300 import binding as B
    rng = np.random.default_rng(3)
    n = 9000
    means = np.stack([rng.uniform(-0.05, 0.05, n), rng.uniform(-0.05, 0.05, n), rng.uniform(2, 6, n)], 1)
    sc = scenes.random_gaussians(rng, means, 0, np.log(0.01), 0.3)
    sc.opacity_logits[:] = -4.0  # keep pixels from saturating so every duplicate is reached
    sc.cameras = [scenes.camera(32, 32, 40.0, 40.0, 15.5, 15.5)]
    gpu = R.render_np(sc, options=_opts(full_lists=1))
    keys, vals, ranges = B.s3gs_debug_binning(R.ctx, R.state)
    assert np.diff(ranges).max() > 4096
    rec = B.s3gs_debug_records(R.ctx, R.state, n)
    qc = B.s3gs_debug_cover(R.ctx, R.state, n)
    rk, rv, rr = O.bin_referee([(32, 32)], 16, 16, rec["xy"][:, 0], rec["xy"][:, 1], rec["extent"][:, 0],
                               rec["extent"][:, 1], rec["rgb_depth"][:, 3], conic=rec["conic_opacity"][:, :3],
                               q_cover=qc)
    assert np.array_equal(keys, rk) and np.array_equal(vals, rv) and np.array_equal(ranges, rr)
    # a deliberately dense stack: more pixels sit near a threshold than in the workloads
    compare_forward(gpu, O.render_fwd(sc), sc.cameras, max_excluded=0.05)


@pytest.mark.parametrize("n_same,n_rest", [(200, 300), (700, 400), (5000, 1000)])
def test_equal_depth_stacks_sort_exactly(R, n_same, n_rest):
    """A stack of Gaussians at one depth fills a single refined depth sub-bin, so
    the tile sort meets one segment longer than a warp network holds (a block
    sort in shared memory, or for more than 4096 keys the chunked global one);
    equal depths must come out by ascending index."""
    from paper_2507_03737_gb300 import binding as B
    rng = np.random.default_rng(n_same)
    n = n_same + n_rest
    z = np.concatenate([np.full(n_same, 3.0), rng.uniform(2, 6, n_rest)])
    means = np.stack([rng.uniform(-0.1, 0.1, n), rng.uniform(-0.1, 0.1, n), z], 1)
    perm = rng.permutation(n)  # interleave the stack with the others in index order
    sc = scenes.random_gaussians(rng, means[perm], 0, np.log(0.01), 0.3)
    sc.cameras = [scenes.camera(32, 32, 40.0, 40.0, 15.5, 15.5)]
    R.render_np(sc, options=_opts(full_lists=1))
    keys, vals, ranges = B.s3gs_debug_binning(R.ctx, R.state)
    rec = B.s3gs_debug_records(R.ctx, R.state, n)
    qc = B.s3gs_debug_cover(R.ctx, R.state, n)
    rk, rv, rr = O.bin_referee([(32, 32)], 16, 16, rec["xy"][:, 0], rec["xy"][:, 1], rec["extent"][:, 0],
                               rec["extent"][:, 1], rec["rgb_depth"][:, 3], conic=rec["conic_opacity"][:, :3],
                               q_cover=qc)
    depth = rec["rgb_depth"][:, 3]
    assert np.count_nonzero(depth == np.float32(3.0)) >= n_same // 2
    assert np.diff(ranges).max() > (4096 if n_same > 4096 else n_same // 2)
    assert np.array_equal(keys, rk) and np.array_equal(vals, rv) and np.array_equal(ranges, rr)


def test_edge_cases(R):
    from paper_2507_03737_gb300 import binding as B
    cam = scenes.camera(20, 10, 20.0, 20.0, 9.5, 4.5)
    # empty scene: background only
    empty = scenes.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
                         np.zeros(0, np.float32), np.zeros((0, 1, 3), np.float32), 0, [cam])
    import torch
    p = {k: torch.zeros((1,) + v.shape[1:], device="cuda")[:0] for k, v in
         dict(means=empty.means, log_scales=empty.log_scales, quats=torch.zeros(0, 4),
              opacity_logits=torch.zeros(0), colors=torch.zeros(0, 1, 3)).items()}
    p["sh_degree"] = 0
    out = R.forward(p, [cam], options=_opts(bg=(0.1, 0.2, 0.3)))
    rgb = out["rgb"].cpu().numpy().reshape(3, -1)
    assert np.allclose(rgb[0], 0.1) and np.allclose(rgb[2], 0.3) and float(out["alpha"].abs().max()) == 0.0
    g = R.backward(p, 1, {"rgb": torch.ones(600, device="cuda")})
    assert float(g["twist"].abs().max()) == 0.0
    # everything behind the camera or beyond the image
    sc = scenes.tiny_scene(12, n=10, width=20, height=10)
    sc.means[:5, 2] = -3.0
    sc.means[5:, 0] = 50.0
    out = R.render_np(sc)
    assert np.abs(out["alpha"]).max() == 0.0
    # one Gaussian filling the view
    one = scenes.tiny_scene(13, n=1, width=24, height=20, scale=2.0)
    compare_forward(R.render_np(one), O.render_fwd(one), one.cameras)


def test_errors_are_reported(R):
    import torch
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.tiny_scene(14, n=50, width=40, height=30)
    p = R.upload(sc)
    st = R.acquire()
    with pytest.raises(B.S3GSError) as e:
        R.backward(p, 1, {}, state=st)
    assert e.value.status == B.S3GS_E_STATE
    for cams, kw, status in (
            ([], {}, B.S3GS_E_INVALID),
            ([sc.cameras[0]] * 33, {}, B.S3GS_E_INVALID),
            (sc.cameras, dict(tile_w=12, tile_h=12), B.S3GS_E_INVALID),
            (sc.cameras, dict(tile_w=8, tile_h=8, pixels_per_thread=4), B.S3GS_E_INVALID),
            (sc.cameras, dict(tile_w=8, tile_h=8, bwd_pixels_per_thread=4), B.S3GS_E_INVALID),
            (sc.cameras, dict(tile_w=8, tile_h=8, pixels_per_thread=2, bwd_pixels_per_thread=8), B.S3GS_E_INVALID),
            (sc.cameras, dict(pixels_per_thread=3), B.S3GS_E_INVALID),
            ([dict(sc.cameras[0], fx=float("nan"))], {}, B.S3GS_E_INVALID),
            ([dict(sc.cameras[0], width=0)], {}, B.S3GS_E_INVALID)):
        with pytest.raises(B.S3GSError) as e:
            R.forward(p, cams if cams else [sc.cameras[0]], options=_opts(**kw), state=st) if cams else \
                B.s3gs_render_fwd(R.ctx, st, B.make_gaussians(p["means"], p["log_scales"], p["quats"],
                                                              p["opacity_logits"], p["colors"], 0),
                                  B.make_cameras(sc.cameras), 0, None, _opts(), None, None, None, None)
        assert e.value.status == status
    bad = dict(p, sh_degree=4)
    with pytest.raises(B.S3GSError):
        R.forward(bad, sc.cameras, state=st)
    # capacity: a tiny reserved duplicate buffer without auto-grow
    st2 = B.s3gs_state_create(R.ctx)
    B.s3gs_reserve(R.ctx, st2, sc.n, 1, 40 * 30, 12, 4)
    R.forward(p, sc.cameras, options=_opts(auto_grow=0), state=st2)
    status, K, cap = B.s3gs_state_check(R.ctx, st2, raise_on_error=False)
    assert status == B.S3GS_E_CAPACITY and K > cap == 4
    # the same state recovers once auto-grow is allowed again
    R.forward(p, sc.cameras, options=_opts(auto_grow=1), state=st2)
    status, K2, cap2 = B.s3gs_state_check(R.ctx, st2, raise_on_error=False)
    assert status == B.S3GS_OK and cap2 >= K2 == K
    B.s3gs_state_destroy(st2)
    R.release(st)
    torch.cuda.synchronize()


def test_mapping_loss_kernel(R):
    import torch
    from paper_2507_03737_gb300 import binding as B
    rng = np.random.default_rng(0)
    cams = [scenes.camera(33, 17, 30, 30, 16, 8), scenes.camera(20, 40, 30, 30, 10, 20)]
    P = 33 * 17 + 20 * 40
    t = lambda a: torch.as_tensor(a.astype(np.float32), device="cuda")
    x = {k: rng.standard_normal(n) for k, n in (("rgb", 3 * P), ("depth", P), ("pm", 3 * P))}
    y = {k: rng.standard_normal(v.size) for k, v in x.items()}
    mask = (rng.uniform(size=P) > 0.3).astype(np.float64)
    d = {k: torch.empty(v.size, device="cuda") for k, v in x.items()}
    loss = torch.zeros(1, device="cuda")
    w = (0.98, 0.5, 0.02)
    B.s3gs_mapping_loss(R.ctx, B.make_cameras(cams), 2, t(x["rgb"]), t(x["depth"]), t(x["pm"]), t(y["rgb"]),
                        t(y["depth"]), t(y["pm"]), t(mask), *w, d["rgb"], d["depth"], d["pm"], loss)
    torch.cuda.synchronize()
    m3 = expand3(mask, cams)
    xr = {k: x[k].astype(np.float32).astype(np.float64) for k in x}
    yr = {k: y[k].astype(np.float32).astype(np.float64) for k in y}
    ref = (w[0] * np.sum(m3 * np.abs(xr["rgb"] - yr["rgb"])) / (3 * P) +
           w[1] * np.sum(mask * np.abs(xr["depth"] - yr["depth"])) / P +
           w[2] * np.sum(m3 * np.abs(xr["pm"] - yr["pm"])) / (3 * P))
    assert abs(float(loss.item()) - ref) < 1e-5 * abs(ref)
    np.testing.assert_allclose(d["rgb"].cpu().numpy(), w[0] * m3 * np.sign(xr["rgb"] - yr["rgb"]) / (3 * P),
                               rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(d["depth"].cpu().numpy(), w[1] * mask * np.sign(xr["depth"] - yr["depth"]) / P,
                               rtol=1e-5, atol=1e-12)


def test_autograd_function_and_pose_gradient(R):
    """torch.autograd drives the CUDA backward; the twist gradient decreases a tracking loss."""
    import torch
    from oracle.pose_oracle import apply_left, se3_exp
    from paper_2507_03737_gb300.autograd import render

    def apply_twist(T, tau):
        return apply_left(se3_exp(tau), np.asarray(T, np.float64))
    sc = scenes.tiny_scene(15, n=200, width=64, height=48, scale=0.15, max_opacity=0.9)
    p = R.upload(sc)
    cam = sc.cameras[0]
    target = [t.detach() for t in render(R, p, [cam])]
    off = dict(cam, T_cw=apply_twist(cam["T_cw"], np.array([0.02, -0.01, 0.0, 0.0, 0.01, -0.01])))
    losses = []
    for it in range(12):
        tw = torch.zeros(1, 6, device="cuda", requires_grad=True)
        rgb, depth, pm, alpha = render(R, p, [off], twist=tw)
        loss = (rgb - target[0]).abs().mean()
        loss.backward()
        losses.append(float(loss.detach()))
        g = tw.grad.detach().cpu().numpy()[0].astype(np.float64)
        off = dict(off, T_cw=apply_twist(off["T_cw"], -2e-3 * g / max(np.linalg.norm(g), 1e-12)))
    assert losses[-1] < losses[0]
    # parameters receive gradients through the same Function
    q = {k: (v.clone().requires_grad_(True) if k != "sh_degree" else v) for k, v in p.items()}
    rgb, depth, pm, alpha = render(R, q, [cam])
    (rgb.sum() + depth.sum()).backward()
    assert float(q["means"].grad.abs().sum()) > 0 and float(q["colors"].grad.abs().sum()) > 0


def test_autotuner_picks_a_valid_schedule_that_keeps_results(R, tmp_path):
    from paper_2507_03737_gb300 import autotune as AT
    sc = scenes.tiny_scene(16, n=2000, width=96, height=64, n_views=2, scale=0.12)
    p = R.upload(sc)
    cache = str(tmp_path / "tune.json")
    best = AT.autotune(R, p, sc.cameras, cache_path=cache, repeats=2, rounds=1)
    assert AT._valid(best)
    import json
    assert AT.signature(p, sc.cameras, best) in json.load(open(cache))
    base = R.render_np(sc)
    tuned = R.render_np(sc, options=best)
    for k in base:
        np.testing.assert_array_equal(tuned[k], base[k])
    again = AT.autotune(R, p, sc.cameras, cache_path=cache)
    assert AT.options_to_dict(again) == AT.options_to_dict(best)


def test_guard_cone_matches_oracle(R):
    """Near-plane, off-axis Gaussians (z 0.21-0.5 m, up to |x/z| = 2.9): culled by the
    guard cone (default) and rendered exactly without it; both against the oracle with
    the same rule. With the cone every gradient tensor is compared. Without it the
    Gaussians just in front of the camera far off-axis are exactly the ill-conditioned
    case the cone exists for (FP32 gradients of their means and of the twist differ
    from FP64 at the 1e-3 level), so there the forward and the colour and opacity
    gradients are compared here, and every tensor on the well-conditioned scene of
    test_no_guard_cone_every_gradient."""
    rng = np.random.default_rng(17)
    n = 40
    means = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.4, 0.4, n), rng.uniform(0.21, 0.5, n)], 1)
    sc = scenes.random_gaussians(rng, means, 0, np.log(0.08), 0.3)
    sc.cameras = [scenes.camera(64, 48, 60.0, 60.0, 31.5, 23.5)]
    try:
        for g in (1.5, -1.0):
            O.set_guard(g)
            ref = O.render_fwd(sc)
            gpu = R.render_np(sc, options=_opts(guard_slope=g))
            compare_forward(gpu, ref, sc.cameras, max_excluded=0.05, name="guard near-plane guard=%g" % g)
            ups = upstream(sc.cameras, 5, pixel_mask(ref))
            g_gpu = R.backward_np(ups, 1)
            g_ref = O.render_bwd(sc, **ups)
            keys = ("means", "log_scales", "quats", "opacity_logits", "colors", "twist") if g > 0 else \
                ("colors", "opacity_logits")
            for k in keys:
                assert rel_l2(g_gpu[k], g_ref[k]) < 1e-3, (g, k, rel_l2(g_gpu[k], g_ref[k]))
    finally:
        O.set_guard(1.5)


def test_no_guard_cone_every_gradient(R):
    """Without the guard cone (the plain definition of the projection), on a
    well-conditioned wide-angle scene: no Gaussian nearer than 1 m, means out to
    |x/z| = 2.4 and |y/z| = 1.8, about half of them outside the default cone. The
    forward and all five parameter tensors and the twist against the oracle without
    the cone, and with it (which culls those Gaussians)."""
    rng = np.random.default_rng(23)
    n = 400
    z = rng.uniform(1.0, 4.0, n)
    means = np.stack([rng.uniform(-2.4, 2.4, n) * z, rng.uniform(-1.8, 1.8, n) * z, z], 1)
    sc = scenes.random_gaussians(rng, means, 0, np.log(0.08), 0.3)
    sc.cameras = [scenes.camera(96, 72, 20.0, 20.0, 47.5, 35.5)]
    outside = (np.abs(means[:, 0] / z) > 1.5) | (np.abs(means[:, 1] / z) > 1.5)
    assert 0.3 * n < outside.sum() < 0.7 * n
    try:
        for g in (-1.0, 1.5):
            O.set_guard(g)
            ref = O.render_fwd(sc)
            gpu = R.render_np(sc, options=_opts(guard_slope=g))
            compare_forward(gpu, ref, sc.cameras, name="no-cone wide guard=%g" % g)
            ups = upstream(sc.cameras, 6, pixel_mask(ref))
            compare_grads(R.backward_np(ups, 1), O.render_bwd(sc, **ups))
    finally:
        O.set_guard(1.5)


def test_pose_only_backward_matches_the_full_twist(R):
    """A backward asking only for the twist (degree-0 colour) accumulates only the
    geometry slots; its twist equals the full backward's up to summation order."""
    sc = scenes.config_scene(1)
    sc2 = scenes.tiny_scene(4, n=200, width=64, height=48, n_views=3)
    for s in (sc, sc2):
        R.render_np(s)
        V = len(s.cameras)
        P = sum(c["width"] * c["height"] for c in s.cameras)
        rng = np.random.default_rng(3)
        ups = dict(d_rgb=rng.standard_normal(3 * P), d_depth=rng.standard_normal(P),
                   d_pointmap=rng.standard_normal(3 * P), d_alpha=rng.standard_normal(P))
        full = R.backward_np(ups, V)
        pose = R.backward_np(ups, V, want=("twist",))
        assert set(pose) == {"twist"}
        np.testing.assert_allclose(pose["twist"], full["twist"], rtol=1e-5,
                                   atol=1e-6 * float(np.abs(full["twist"]).max()))


@pytest.mark.parametrize("det,masked,terms", [(1, False, "all"), (0, True, "all"), (1, True, "rgb_geo")])
def test_fused_loss_backward_matches_loss_then_backward(R, det, masked, terms):
    """s3gs_render_bwd_l1 equals s3gs_mapping_loss followed by s3gs_render_bwd: same
    gradients (deterministic mode: up to FP32 contraction order of the pointmap term,
    1e-6 relative per tensor; atomic mode: summation order, 1e-5), loss within 1e-5."""
    import torch
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.tiny_scene(7, n=300, width=77, height=45, n_views=3, scale=0.2)
    sc.cameras[1] = dict(sc.cameras[1], width=33, height=70)
    tgt_sc = scenes.perturb_scene(sc, 9, sigma_pos=0.05, sigma_col=0.1)
    opt = B.s3gs_options_default(deterministic=det)
    p_t = R.upload(tgt_sc)
    tgt = {k: v.clone() for k, v in R.forward(p_t, sc.cameras, options=opt).items()}
    p = R.upload(sc)
    P = sum(c["width"] * c["height"] for c in sc.cameras)
    mask = torch.from_numpy(np.random.default_rng(2).uniform(0, 1, P).astype(np.float32)).cuda() if masked else None
    t_depth = tgt["depth"] if terms == "all" else None
    cams = B.make_cameras(sc.cameras)

    def grads():
        return {k: torch.zeros_like(p[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "colors")} | \
            {"twist": torch.zeros((3, 6), device="cuda")}
    out = R.forward(p, sc.cameras, options=opt)
    d = {k: torch.empty_like(out[k]) for k in ("rgb", "depth", "pointmap")}
    loss_a = torch.zeros(1, device="cuda")
    B.s3gs_mapping_loss(R.ctx, cams, 3, out["rgb"], out["depth"], out["pointmap"], tgt["rgb"], t_depth,
                        tgt["pointmap"], mask, 0.98, 0.02, 0.02, d["rgb"], d["depth"], d["pointmap"], loss_a)
    ga = grads()
    B.s3gs_render_bwd(R.ctx, R.state, d["rgb"], d["depth"], d["pointmap"], None, ga["means"], ga["log_scales"],
                      ga["quats"], ga["opacity_logits"], ga["colors"], ga["twist"], 0)
    out2 = R.forward(p, sc.cameras, options=opt)
    gb = grads()
    loss_b = torch.zeros(1, device="cuda")
    B.s3gs_render_bwd_l1(R.ctx, R.state, out2["rgb"], out2["depth"], out2["pointmap"], tgt["rgb"], t_depth,
                         tgt["pointmap"], mask, 0.98, 0.02, 0.02, loss_b, gb["means"], gb["log_scales"], gb["quats"],
                         gb["opacity_logits"], gb["colors"], gb["twist"], 0)
    torch.cuda.synchronize()
    tol = 1e-6 if det else 1e-5
    for k in ga:
        a, b = ga[k].cpu().numpy().astype(np.float64), gb[k].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - b) <= tol * max(np.linalg.norm(a), 1e-30), k
    assert abs(float(loss_a[0]) - float(loss_b[0])) <= 1e-5 * abs(float(loss_a[0]))
