"""The headline window step as the benchmark times it, and the autograd Function.

1. The step the benchmark replays -- s3gs_render_fwd followed by
   s3gs_render_bwd_l1 (Eq. 10/15/17 fused into the backward) -- captured in a
   CUDA graph: each replay equals the eager step bit for bit in deterministic
   mode, and both equal the FP64 oracle (outputs, loss, every gradient tensor and
   the twist) on config 1.
2. torch.autograd through RenderFunction: every parameter gradient and the twist
   gradient against the oracle's analytic gradient (Sec. 3.2.2, Eq. 11) per
   tensor at 1e-3, and a directional derivative of the loss against central
   finite differences of the GPU's own forward.
"""
import numpy as np
import pytest

import oracle as O
from oracle.pose_oracle import apply_left, se3_exp
from paper_2507_03737_gb300 import scenes
from tests.gpu_helpers import compare_forward, compare_grads, expand3, pixel_mask, upstream

pytestmark = pytest.mark.gpu

W_RGB, W_DEPTH, W_GEO = 0.98, 0.02, 0.02
PARAMS = ("means", "log_scales", "quats", "opacity_logits", "colors")


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2507_03737_gb300.autograd import Renderer
    r = Renderer(0)
    yield r
    r.close()


def _l1_reference(sc, ref, tgt, mask):
    """FP64 loss and upstream gradients of the mapping loss (Eq. 17 with a depth term;
    means over the elements of each term, per-pixel weight ``mask``)."""
    cams = sc.cameras
    P = sum(c["width"] * c["height"] for c in cams)
    m3 = expand3(mask, cams)
    r_rgb = ref["rgb"] - tgt["rgb"]
    r_d = ref["depth"] - tgt["depth"]
    r_pm = ref["pointmap"] - tgt["pointmap"]
    loss = (W_RGB * np.sum(m3 * np.abs(r_rgb)) / (3 * P) + W_DEPTH * np.sum(mask * np.abs(r_d)) / P +
            W_GEO * np.sum(m3 * np.abs(r_pm)) / (3 * P))
    ups = dict(d_rgb=W_RGB * m3 * np.sign(r_rgb) / (3 * P), d_depth=W_DEPTH * mask * np.sign(r_d) / P,
               d_pointmap=W_GEO * m3 * np.sign(r_pm) / (3 * P))
    return loss, ups


@pytest.mark.parametrize("schedule", [{}, dict(tile_w=8, tile_h=8, pixels_per_thread=1, bwd_pixels_per_thread=1,
                                                batch=64), dict(blocks_per_sm=12, pixels_per_thread=2,
                                                                bwd_pixels_per_thread=4, batch=128)],
                         ids=["default", "config1_tuned", "config3_tuned"])
def test_window_step_graph_replay_equals_eager_and_oracle(R, schedule):
    import torch
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.config_scene(1)
    cams = sc.cameras
    P = sum(c["width"] * c["height"] for c in cams)
    opt = B.s3gs_options_default(deterministic=1, **schedule)
    tgt_t = {k: v.clone() for k, v in R.forward(R.upload(scenes.perturb_scene(sc, 77)), cams, options=opt).items()}
    torch.cuda.synchronize()
    tgt = {k: v.cpu().numpy().astype(np.float64) for k, v in tgt_t.items()}
    ref = O.render_fwd(sc)
    # the loss weight masks out pixels whose FP64 decisions sit near a threshold and
    # pixels where a residual is within the forward tolerance of zero (the L1 sign)
    clear = pixel_mask(ref)
    near0 = np.zeros(P, bool)
    for k, ch in (("rgb", 3), ("pointmap", 3), ("depth", 1)):
        r = (ref[k] - tgt[k]).reshape(ch, P)
        near0 |= (np.abs(r) <= 3e-4 * (np.abs(ref[k].reshape(ch, P)) + 1.0)).any(0)
    near0 &= (np.abs(ref["alpha"]) > 0) | (np.abs(tgt["alpha"]) > 0)  # empty in both: residual exactly 0
    mask = (clear & ~near0).astype(np.float64)
    assert mask.sum() > 0.8 * P
    mask_t = torch.as_tensor(mask.astype(np.float32), device="cuda")

    p = R.upload(sc)
    gs = B.make_gaussians(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["colors"], 0)
    cam_arr = B.make_cameras(cams)
    out = R.empty_outputs(cams)
    grads = {k: torch.zeros_like(p[k]) for k in PARAMS} | {"twist": torch.zeros((1, 6), device="cuda")}
    loss = torch.zeros(1, device="cuda")

    def step():
        B.s3gs_render_fwd(R.ctx, R.state, gs, cam_arr, 1, None, opt, out["rgb"], out["depth"], out["pointmap"],
                          out["alpha"])
        B.s3gs_render_bwd_l1(R.ctx, R.state, out["rgb"], out["depth"], out["pointmap"], tgt_t["rgb"],
                             tgt_t["depth"], tgt_t["pointmap"], mask_t, W_RGB, W_DEPTH, W_GEO, loss,
                             grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logits"],
                             grads["colors"], grads["twist"], 0)

    def snapshot():
        torch.cuda.synchronize()
        return {k: v.cpu().numpy().copy() for k, v in (out | grads | {"loss": loss}).items()}

    step()
    eager = snapshot()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        for t in list(out.values()) + list(grads.values()) + [loss]:
            t.fill_(float("nan"))  # the replay must write every output it owns
        graph.replay()
        replay = snapshot()
        for k in eager:
            np.testing.assert_array_equal(replay[k], eager[k], err_msg=k)
    # both against the oracle
    compare_forward({k: eager[k] for k in ("rgb", "depth", "pointmap", "alpha")}, ref, cams)
    loss64, ups = _l1_reference(sc, ref, tgt, mask)
    assert abs(float(eager["loss"][0]) - loss64) <= 1e-5 * abs(loss64), (float(eager["loss"][0]), loss64)
    gref = O.render_bwd(sc, **ups)
    compare_grads({k: eager[k] for k in PARAMS + ("twist",)}, gref)


def _params(R, sc, twist_views):
    import torch
    p = R.upload(sc)
    q = {k: (v.clone().requires_grad_(True) if k != "sh_degree" else v) for k, v in p.items()}
    tw = torch.zeros((twist_views, 6), device="cuda", requires_grad=True)
    return q, tw


def _weighted_loss(outs, ups_t):
    rgb, depth, pm, alpha = outs
    return ((rgb * ups_t["d_rgb"]).sum() + (depth * ups_t["d_depth"]).sum() + (pm * ups_t["d_pointmap"]).sum() +
            (alpha * ups_t["d_alpha"]).sum())


@pytest.mark.parametrize("case", ["config1", "sh3_two_views"])
def test_autograd_function_gradients_match_oracle(R, case):
    """loss = sum(d_out * out) through RenderFunction: each .grad against the oracle's
    gradient of the same loss, per tensor, twist included."""
    import torch
    from paper_2507_03737_gb300.autograd import render
    if case == "config1":
        sc = scenes.config_scene(1)
    else:
        sc = scenes.tiny_scene(71, n=60, width=48, height=36, sh_degree=3, n_views=2, scale=0.2)
    cams = sc.cameras
    ref = O.render_fwd(sc)
    ups = upstream(cams, 13, pixel_mask(ref))
    ups_t = {k: torch.as_tensor(v.astype(np.float32), device="cuda") for k, v in ups.items()}
    q, tw = _params(R, sc, len(cams))
    outs = render(R, q, cams, twist=tw)
    compare_forward({k: o.detach().cpu().numpy() for k, o in zip(("rgb", "depth", "pointmap", "alpha"), outs)},
                    ref, cams)
    _weighted_loss(outs, ups_t).backward()
    got = {k: q[k].grad.cpu().numpy() for k in PARAMS} | {"twist": tw.grad.cpu().numpy()}
    gref = O.render_bwd(sc, **ups)
    compare_grads(got, gref)


def test_autograd_directional_derivative_matches_finite_differences(R):
    """<grad L, delta> from the autograd backward against (L(x + h delta) - L(x - h delta)) / 2h
    of the GPU's own forward, for random directions in the means, the colours and the
    twist (the pose moved by Exp(+-h tau) T_cw), one at a time.

    A pixel's outputs depend only on the decisions taken at that pixel. Opacities of
    at least 0.4 keep the 1/255 skip from binding inside the 3-sigma ellipse, upstream
    weights vanish wherever the oracle reports a decision within 2e-3 of its threshold
    (it reports every decision within 1e-3 exactly), and a step of 5e-5 moves q by
    well under 1e-3 relative, so no decision of a weighted pixel flips between the two
    evaluations; the FP64 oracle's own difference quotient at the same step is checked
    against its analytic derivative first to show it. The loss of each GPU forward is
    summed in FP64 on the host; its FP32 outputs bound the agreement near 1e-3."""
    import torch
    from paper_2507_03737_gb300.autograd import render
    sc = scenes.tiny_scene(72, n=12, width=40, height=32, scale=0.3, max_opacity=0.8)
    op = np.random.default_rng(72).uniform(0.4, 0.8, sc.n)
    sc.opacity_logits = np.log(op / (1 - op)).astype(np.float32)
    cam = sc.cameras[0]
    P = 40 * 32
    ref = O.render_fwd(sc)
    smooth = ref["margin"] > 2e-3
    assert smooth.sum() > 0.5 * P
    rng = np.random.default_rng(5)
    m3 = np.tile(smooth, 3)
    ups = dict(d_rgb=rng.standard_normal(3 * P) * m3, d_depth=rng.standard_normal(P) * 0.1 * smooth,
               d_pointmap=rng.standard_normal(3 * P) * 0.1 * m3, d_alpha=rng.standard_normal(P) * smooth)
    ups_t = {k: torch.as_tensor(v.astype(np.float32), device="cuda") for k, v in ups.items()}
    q, tw = _params(R, sc, 1)
    _weighted_loss(render(R, q, [cam], twist=tw), ups_t).backward()
    d = dict(means=rng.standard_normal(sc.means.shape), colors=rng.standard_normal(sc.colors.shape),
             twist=rng.standard_normal(6) * np.array([1, 1, 1, 0.3, 0.3, 0.3]))
    gpu_grad = dict(means=q["means"].grad.cpu().numpy(), colors=q["colors"].grad.cpu().numpy(),
                    twist=tw.grad.cpu().numpy()[0])
    gref = O.render_bwd(sc, **ups)
    gref["twist"] = gref["twist"][0]

    def moved(s, which):
        out = sc.subset(slice(None))
        c = cam
        if which == "means":
            out.means = sc.means.astype(np.float64) + s * d["means"]
        elif which == "colors":
            out.colors = sc.colors.astype(np.float64) + s * d["colors"]
        else:
            c = dict(cam, T_cw=apply_left(se3_exp(s * d["twist"]), np.asarray(cam["T_cw"], np.float64)))
        return out, c

    def loss_gpu(s, which):
        sc2, c = moved(s, which)
        p = R.upload(sc2)
        c = dict(c, T_cw=np.asarray(c["T_cw"], np.float32))
        with torch.no_grad():
            outs = [o.double().cpu().numpy() for o in render(R, p, [c])]
        return sum(float(np.dot(o, ups[k])) for o, k in zip(outs, ("d_rgb", "d_depth", "d_pointmap", "d_alpha")))

    def loss_oracle(s, which):
        sc2, c = moved(s, which)
        f = O.render_fwd(sc2, cameras=[c])
        return sum(float(np.dot(f[k], ups["d_" + k])) for k in ("rgb", "depth", "pointmap", "alpha"))

    # the render is linear in degree-0 colours, so their step can be large
    for which, h, least in (("means", 5e-5, 1.0), ("colors", 1e-2, 1e-2), ("twist", 5e-5, 1.0)):
        analytic = float((gpu_grad[which] * d[which]).sum())
        analytic64 = float((gref[which] * d[which]).sum())
        fd64 = (loss_oracle(h, which) - loss_oracle(-h, which)) / (2 * h)
        assert abs(fd64 - analytic64) <= 1e-5 * abs(analytic64), (which, "oracle", fd64, analytic64)
        fd = (loss_gpu(h, which) - loss_gpu(-h, which)) / (2 * h)
        assert abs(analytic) > least, (which, analytic)
        assert abs(fd - analytic) <= 5e-3 * abs(analytic), (which, fd, analytic)
