"""PyTorch front end: a renderer handle and a ``torch.autograd.Function``.

The forward and backward both run in ``libs3gs.so``. The camera twist enters
as an extra input ``twist`` of shape (n_views, 6), a perturbation tau =
(rho, phi) applied as Exp(tau) * T_cw; the forward renders at tau = 0 (its
value is not read) and the backward returns dL/dtau there (Sec. 3.2.2, Eq. 11),
which is what a pose-refinement step needs.
"""
from __future__ import annotations

import weakref

import numpy as np
import torch

from . import binding as B

__all__ = ["Renderer", "RenderFunction", "render", "OUTPUTS"]

OUTPUTS = ("rgb", "depth", "pointmap", "alpha")
PARAMS = ("means", "log_scales", "quats", "opacity_logits", "colors")


def _n_pixels(cameras):
    return sum(int(c["width"]) * int(c["height"]) for c in cameras)


class Renderer:
    """Owns one library context on a device and a pool of forward states."""

    def __init__(self, device: int = 0, options: B.Options | None = None):
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.ctx = B.s3gs_create(device)
        self.options = options if options is not None else B.s3gs_options_default()
        self._free = []
        self._all = []
        self.state = self.acquire()

    # ---- state pool ----
    def acquire(self):
        if self._free:
            return self._free.pop()
        s = B.s3gs_state_create(self.ctx)
        self._all.append(s)
        return s

    def release(self, state):
        if state in self._all and state not in self._free:
            self._free.append(state)

    def close(self):
        if self.ctx is None:
            return
        torch.cuda.synchronize(self.device)
        for s in self._all:
            B.s3gs_state_destroy(s)
        self._all.clear()
        self._free.clear()
        B.s3gs_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- tensors ----
    def upload(self, scene) -> dict:
        dev = self.device
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
        return dict(means=t(scene.means), log_scales=t(scene.log_scales), quats=t(scene.quats),
                    opacity_logits=t(scene.opacity_logits), colors=t(scene.colors),
                    sh_degree=int(scene.sh_degree))

    def empty_outputs(self, cameras, which=OUTPUTS) -> dict:
        P = _n_pixels(cameras)
        sizes = dict(rgb=3 * P, depth=P, pointmap=3 * P, alpha=P)
        return {k: torch.empty(sizes[k], device=self.device, dtype=torch.float32) for k in which}

    def forward(self, params: dict, cameras, options=None, state=None, T_cw_device=None,
                outputs=None, which=OUTPUTS, stream=None) -> dict:
        state = self.state if state is None else state
        out = outputs if outputs is not None else self.empty_outputs(cameras, which)
        g = B.make_gaussians(params["means"], params["log_scales"], params["quats"],
                             params["opacity_logits"], params["colors"], params["sh_degree"])
        cams = B.make_cameras(cameras)
        B.s3gs_render_fwd(self.ctx, state, g, cams, len(cameras), T_cw_device,
                          options if options is not None else self.options,
                          out.get("rgb"), out.get("depth"), out.get("pointmap"), out.get("alpha"), stream)
        return out

    def backward(self, params: dict, n_views: int, grads: dict, state=None, want=PARAMS + ("twist",),
                 accumulate=False, into=None, stream=None) -> dict:
        state = self.state if state is None else state
        res = into if into is not None else {}
        if into is None:
            for k in want:
                if k == "twist":
                    res[k] = torch.empty((n_views, 6), device=self.device, dtype=torch.float32)
                else:
                    res[k] = torch.empty_like(params[k])
        B.s3gs_render_bwd(self.ctx, state, grads.get("rgb"), grads.get("depth"), grads.get("pointmap"),
                          grads.get("alpha"), res.get("means"), res.get("log_scales"), res.get("quats"),
                          res.get("opacity_logits"), res.get("colors"), res.get("twist"),
                          int(accumulate), stream)
        return res

    # ---- numpy conveniences for tests ----
    def render_np(self, scene, cameras=None, options=None, state=None) -> dict:
        cameras = scene.cameras if cameras is None else cameras
        p = self.upload(scene)
        out = self.forward(p, cameras, options=options, state=state)
        torch.cuda.synchronize(self.device)
        self._last_params = p
        return {k: v.cpu().numpy() for k, v in out.items()}

    def backward_np(self, ups: dict, n_views: int, state=None, want=PARAMS + ("twist",)) -> dict:
        dev = self.device
        g = {k[2:] if k.startswith("d_") else k: torch.as_tensor(np.asarray(v, np.float32), device=dev)
             for k, v in ups.items() if v is not None}
        res = self.backward(self._last_params, n_views, g, state=state, want=want)
        torch.cuda.synchronize(dev)
        return {k: v.cpu().numpy() for k, v in res.items()}

    def render_and_backward_np(self, scene, seed=0):
        out = self.render_np(scene)
        P = _n_pixels(scene.cameras)
        rng = np.random.default_rng(seed)
        ups = dict(d_rgb=rng.standard_normal(3 * P), d_depth=rng.standard_normal(P),
                   d_pointmap=rng.standard_normal(3 * P), d_alpha=rng.standard_normal(P))
        grads = self.backward_np(ups, len(scene.cameras))
        return out, grads


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, colors, twist, renderer, cameras,
                sh_degree, options):
        state = renderer.acquire()
        params = dict(means=means.detach().contiguous(), log_scales=log_scales.detach().contiguous(),
                      quats=quats.detach().contiguous(), opacity_logits=opacity_logits.detach().contiguous(),
                      colors=colors.detach().contiguous(), sh_degree=int(sh_degree))
        out = renderer.forward(params, cameras, options=options, state=state)
        ctx.renderer = renderer
        ctx.state = state
        ctx.params = params
        ctx.n_views = len(cameras)
        ctx.needs = ctx.needs_input_grad
        weakref.finalize(ctx, renderer.release, state)
        return out["rgb"], out["depth"], out["pointmap"], out["alpha"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_pointmap, g_alpha):
        grads = {}
        for k, g in zip(OUTPUTS, (g_rgb, g_depth, g_pointmap, g_alpha)):
            if g is not None:
                grads[k] = g.contiguous()
        want = tuple(k for k, need in zip(PARAMS + ("twist",), ctx.needs[:6]) if need)
        res = ctx.renderer.backward(ctx.params, ctx.n_views, grads, state=ctx.state, want=want)
        ctx.renderer.release(ctx.state)
        out = [res.get(k) for k in PARAMS + ("twist",)]
        return (*out, None, None, None, None)


def render(renderer: Renderer, params: dict, cameras, twist=None, options=None):
    """Differentiable render; returns (rgb, depth, pointmap, alpha) packed tensors."""
    if twist is None:
        twist = torch.zeros((len(cameras), 6), device=renderer.device, dtype=torch.float32)
    return RenderFunction.apply(params["means"], params["log_scales"], params["quats"],
                                params["opacity_logits"], params["colors"], twist, renderer, cameras,
                                params["sh_degree"], options)

