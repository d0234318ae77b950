"""The fused map-optimiser step (Eq. 16/17) against the FP64 oracle, and the
captured window-mapping iteration.

Tolerances: the step is elementwise FP32 (one division of the bias-corrected
moments, one square root): moments within 1e-5 relative or 1e-5 of the
tensor's largest entry (the first moment sums terms of either sign, and the
log-scale gradient adds an L_iso term that can cancel the input gradient),
parameters within
1e-6 absolute plus 1e-6 relative after four steps (parameters are O(1), steps
O(lr)). The L_iso sign decisions are FP32 on the GPU; the inputs keep every
scale at least 1e-4 (relative) from its Gaussian's mean scale, where FP32 and
FP64 could disagree. The oracle is given the float32 hyperparameters the kernel
receives (0.999f is not 0.999: 1 - beta2 differs by 1.3e-5 relative).
"""
import numpy as np
import pytest

from oracle import adam_oracle as A
from paper_2507_03737_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2507_03737_gb300.autograd import Renderer
    r = Renderer(0)
    yield r
    r.close()


def _random_params(rng, n, sh):
    nc = (sh + 1) ** 2
    ls = rng.normal(-3, 0.6, (n, 3)).astype(np.float32)
    # keep every scale at least 1e-4 (relative) from its Gaussian's mean scale,
    # clear of the L_iso sign decision that FP32 and FP64 could take differently
    while True:
        s = np.exp(ls.astype(np.float64))
        rel = np.abs(s - s.mean(axis=1, keepdims=True)) / s.mean(axis=1, keepdims=True)
        bad = (rel < 1e-4).any(axis=1)
        if not bad.any():
            break
        ls[bad] = rng.normal(-3, 0.6, (int(bad.sum()), 3)).astype(np.float32)
    return dict(means=rng.normal(0, 2, (n, 3)).astype(np.float32),
                log_scales=ls,
                quats=rng.normal(0, 1, (n, 4)).astype(np.float32),
                opacity_logits=rng.normal(0, 1, n).astype(np.float32),
                colors=rng.normal(0, 0.3, (n, nc, 3)).astype(np.float32))


@pytest.mark.parametrize("sh,missing", [(0, ()), (3, ()), (1, ("quats", "colors"))])
def test_map_adam_step_matches_oracle(R, sh, missing):
    import torch
    from paper_2507_03737_gb300 import binding as B
    rng = np.random.default_rng(10 + sh)
    n = 5000
    host = _random_params(rng, n, sh)
    dev = {k: torch.from_numpy(v.copy()).cuda() for k, v in host.items()}
    dev["sh_degree"] = sh
    m = {k: torch.zeros_like(dev[k]) for k in B.MAP_TENSORS}
    v = {k: torch.zeros_like(dev[k]) for k in B.MAP_TENSORS}
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    hp = B.s3gs_map_adam_default(eps=1e-8)
    lrs = dict(means=hp.lr_means, log_scales=hp.lr_log_scales, quats=hp.lr_quats, opacity_logits=hp.lr_opacity,
               colors=hp.lr_colors)
    ref_p = {k: x.astype(np.float64) for k, x in host.items()}
    ref_s = {}
    for t in range(1, 5):
        grads = {k: (rng.normal(0, 1, x.shape) * 10.0 ** rng.uniform(-3, 0)).astype(np.float32)
                 for k, x in host.items()}
        for k in missing:
            grads[k] = np.zeros_like(grads[k])
        dg = {k: torch.from_numpy(x).cuda() for k, x in grads.items() if k not in missing}
        B.s3gs_map_adam_step(R.ctx, dev, dg, m, v, step, hp)
        # the oracle takes the hyperparameters the kernel received (float32 values)
        ref_p, ref_s = A.map_step(ref_p, grads, ref_s, t, lrs, lambda_iso=hp.lambda_iso, beta1=hp.beta1,
                                  beta2=hp.beta2, eps=hp.eps, lr_colors_rest=hp.lr_colors_rest)
        torch.cuda.synchronize()
        for k in B.MAP_TENSORS:
            np.testing.assert_allclose(dev[k].cpu().numpy(), ref_p[k], rtol=1e-6, atol=1e-6, err_msg=k)
            # m = beta1 m + (1 - beta1) g can cancel: its error scales with the terms, not the result
            np.testing.assert_allclose(m[k].cpu().numpy(), ref_s[k][0], rtol=1e-5,
                                       atol=1e-5 * float(np.abs(ref_s[k][0]).max()), err_msg=k)
            # the log-scale gradient adds the L_iso term, which can cancel the input gradient:
            # both moments are checked against the scale of their largest entry as well
            np.testing.assert_allclose(v[k].cpu().numpy(), ref_s[k][1], rtol=1e-5,
                                       atol=1e-5 * float(np.abs(ref_s[k][1]).max()), err_msg=k)
    assert int(step[0]) == 4


def test_iso_alone_drives_scales_toward_isotropy(R):
    import torch
    from paper_2507_03737_gb300 import binding as B
    rng = np.random.default_rng(3)
    host = _random_params(rng, 2000, 0)
    dev = {k: torch.from_numpy(v.copy()).cuda() for k, v in host.items()}
    dev["sh_degree"] = 0
    m = {k: torch.zeros_like(dev[k]) for k in B.MAP_TENSORS}
    v = {k: torch.zeros_like(dev[k]) for k in B.MAP_TENSORS}
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    hp = B.s3gs_map_adam_default(lr_log_scales=1e-2)
    before = A.iso_loss(host["log_scales"])
    for _ in range(50):
        B.s3gs_map_adam_step(R.ctx, dev, {}, m, v, step, hp)
    torch.cuda.synchronize()
    assert A.iso_loss(dev["log_scales"].cpu().numpy()) < 0.5 * before
    # with no gradient and zero moments the other tensors do not move
    assert torch.equal(dev["means"], torch.from_numpy(host["means"]).cuda())


def test_step_replays_from_a_graph(R):
    import torch
    from paper_2507_03737_gb300 import binding as B
    rng = np.random.default_rng(4)
    host = _random_params(rng, 3000, 1)
    grads = {k: torch.from_numpy(rng.normal(0, 0.1, x.shape).astype(np.float32)).cuda() for k, x in host.items()}
    hp = B.s3gs_map_adam_default()

    def fresh():
        d = {k: torch.from_numpy(v.copy()).cuda() for k, v in host.items()}
        d["sh_degree"] = 1
        return d, {k: torch.zeros_like(d[k]) for k in B.MAP_TENSORS}, \
            {k: torch.zeros_like(d[k]) for k in B.MAP_TENSORS}, torch.zeros(1, dtype=torch.int32, device="cuda")
    d1, m1, v1, s1 = fresh()
    for _ in range(3):
        B.s3gs_map_adam_step(R.ctx, d1, grads, m1, v1, s1, hp)
    d2, m2, v2, s2 = fresh()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=st):
        B.s3gs_map_adam_step(R.ctx, d2, grads, m2, v2, s2, hp)
    for k in B.MAP_TENSORS:  # capture does not run the step; restore nothing
        assert torch.equal(d2[k], torch.from_numpy(host[k]).cuda())
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert int(s2[0]) == 3
    for k in B.MAP_TENSORS:
        assert torch.equal(d1[k], d2[k]) and torch.equal(m1[k], m2[k]) and torch.equal(v1[k], v2[k])


def test_window_mapping_iterations_reduce_the_loss(R):
    """Config 1 map against the renders of a perturbed copy: twenty captured
    mapping iterations (render, loss, backward, Adam + L_iso, pose step)."""
    import torch
    from paper_2507_03737_gb300 import binding as B
    from paper_2507_03737_gb300.slam import MapOptimizer
    sc = scenes.config_scene(1)
    tgt_scene = scenes.perturb_scene(sc, 5, sigma_pos=0.05, sigma_col=0.1)
    p_t = R.upload(tgt_scene)
    tgt = R.forward(p_t, sc.cameras)
    t_rgb, t_pm = tgt["rgb"].clone(), tgt["pointmap"].clone()
    p = R.upload(sc)
    hp = B.s3gs_map_adam_default(lambda_iso=10.0 / (3 * sc.n))
    mo = MapOptimizer(R, p, sc.cameras, t_rgb, t_pointmap=t_pm, hp=hp, iters=20,
                      frozen=torch.ones(1, dtype=torch.uint8, device="cuda"))
    mo.iteration()
    torch.cuda.synchronize()
    first = float(mo.loss[0])
    mo.run()
    torch.cuda.synchronize()
    mo.check()
    last = float(mo.loss[0])
    assert last < 0.8 * first, (first, last)
    T0 = np.asarray(sc.cameras[0]["T_cw"], np.float32).reshape(12)
    assert np.array_equal(mo.T.cpu().numpy()[0], T0)  # frozen pose
