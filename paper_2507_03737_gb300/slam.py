"""PyTorch front end of the SLAM steps that consume the rendered pointmap:
patch-based scale alignment (Sec. 3.3.1, Algorithm 1 of the supplementary
material), pointmap replacement (Eq. 14) and the remedial scale factor.

Argument marshalling only; every step runs in ``libs3gs.so`` (C ABI in
``include/s3gs_slam.h``). Pointmaps use the renderer's packed planar layout:
view after view, each [3][H][W].
"""
from __future__ import annotations

import torch

from . import binding as B

__all__ = ["Aligner", "PoseRefiner", "MapOptimizer", "EPS_M"]

EPS_M = 0.15  # Eq. 14 threshold used for all datasets (supplementary material)


class Aligner:
    """Holds a library context (its own, or a renderer's) and a workspace."""

    def __init__(self, ctx=None, device: int = 0):
        self.device = torch.device("cuda", device)
        self._own = ctx is None
        self.ctx = B.s3gs_create(device) if ctx is None else ctx
        self._ws = torch.empty(0, dtype=torch.uint8, device=self.device)

    def close(self):
        if self._own and self.ctx is not None:
            torch.cuda.synchronize(self.device)
            B.s3gs_destroy(self.ctx)
        self.ctx = None

    def workspace(self, wh, nv, patch):
        need = B.s3gs_scale_align_workspace(wh, nv, patch)
        if self._ws.numel() < need:
            self._ws = torch.empty(max(need, 16), dtype=torch.uint8, device=self.device)
        return self._ws

    def align(self, X_r, X_p, views, params: B.AlignParams | None = None, sigma_init=None, want_mask=False,
              out=None, stream=None) -> dict:
        """Algorithm 1 on every view. ``views``: camera dicts or (w, h) pairs."""
        params = params if params is not None else B.s3gs_align_params_default()
        wh, nv = B.view_sizes(views)
        ws = self.workspace(wh, nv, params.patch)
        dev = self.device
        if out is None:
            P = sum(wh[2 * v] * wh[2 * v + 1] for v in range(nv))
            out = dict(sigma=torch.empty(nv, device=dev), n_cp=torch.empty(nv, dtype=torch.int64, device=dev),
                       insufficient=torch.empty(nv, dtype=torch.int32, device=dev),
                       cp_mask=torch.empty(P, dtype=torch.uint8, device=dev) if want_mask else None)
        B.s3gs_scale_align(self.ctx, wh, nv, X_r, X_p, params, sigma_init, out["sigma"], out["n_cp"],
                           out["insufficient"], out.get("cp_mask"), ws, stream)
        return out

    def replace(self, X_r, X_p, sigma, views, eps_m: float = EPS_M, out=None, want_xp_hat=True, want_mask=True,
                stream=None) -> dict:
        """Eq. 14 with Xhat^p = sigma_v X^p."""
        wh, nv = B.view_sizes(views)
        dev = self.device
        if out is None:
            out = dict(X_r_hat=torch.empty_like(X_r), X_p_hat=torch.empty_like(X_p) if want_xp_hat else None,
                       replaced=torch.empty(X_r.numel() // 3, dtype=torch.uint8, device=dev) if want_mask else None,
                       n_replaced=torch.empty(nv, dtype=torch.int64, device=dev))
        B.s3gs_pointmap_replace(self.ctx, wh, nv, X_r, X_p, sigma, eps_m, out["X_r_hat"], out.get("X_p_hat"),
                                out.get("replaced"), out.get("n_replaced"), stream)
        return out

    def remedy(self, X_ak_hat, X_n, matches, stream=None):
        """Remedial factor from matched pixels (device int32 [M][2] flat pixel indices)."""
        sigma = torch.empty(1, device=self.device)
        n_used = torch.empty(1, dtype=torch.int64, device=self.device)
        m = matches.to(device=self.device, dtype=torch.int32).contiguous()
        B.s3gs_scale_remedy(self.ctx, X_ak_hat, X_ak_hat.numel() // 3, X_n, X_n.numel() // 3, m, m.shape[0], sigma,
                            n_used, stream)
        return sigma, n_used

    def align_with_remedy(self, X_r, X_p, views, params=None, remedy=None) -> dict:
        """Algorithm 1, then, for every view whose correct points are too few and
        for which ``remedy[v] = (X_ak_hat, matches)`` is given, the remedial
        factor followed by one more alignment iteration started from it; that
        iteration's factor is the view's result (the supplementary material's
        procedure). Reads the insufficiency flags on the host."""
        params = params if params is not None else B.s3gs_align_params_default()
        res = self.align(X_r, X_p, views, params)
        if not remedy:
            return res
        flags = res["insufficient"].cpu().tolist()
        sizes = [(int(c["width"]), int(c["height"])) if isinstance(c, dict) else (int(c[0]), int(c[1]))
                 for c in views]
        off = 0
        one = B.AlignParams.from_buffer_copy(params)
        one.max_iter = 1
        for v, (w, h) in enumerate(sizes):
            sl = slice(3 * off, 3 * (off + w * h))
            off += w * h
            if not flags[v] or v not in remedy:
                continue
            X_ak_hat, matches = remedy[v]
            s_rem, _ = self.remedy(X_ak_hat, X_p[sl], matches)
            r = self.align(X_r[sl], X_p[sl], [(w, h)], one, sigma_init=s_rem)
            res["sigma"][v] = r["sigma"][0]
            res["n_cp"][v] = r["n_cp"][0]
            res["insufficient"][v] = r["insufficient"][0]
        return res


class PoseRefiner:
    """Photometric pose refinement (Sec. 3.2.2, Eq. 10/11) of one or more views
    against a fixed Gaussian map, entirely on the device: each iteration renders
    at the current poses (``T_cw_device``), evaluates the weighted L1 photometric
    loss, runs the pose-only backward and takes one Adam step with retraction.
    ``capture()`` records the reset to the initial poses plus ``iters``
    iterations into one CUDA graph, so ``run()`` is a single graph launch."""

    def __init__(self, renderer, params: dict, cameras, target_rgb, weight=None, hp: B.PoseAdam | None = None,
                 iters: int = 10, options: B.Options | None = None):
        import numpy as np
        self.R = renderer
        self.params = params
        self.cameras = [dict(c) for c in cameras]
        self.V = len(cameras)
        dev = renderer.device
        self.hp = hp if hp is not None else B.s3gs_pose_adam_default()
        self.iters = int(iters)
        self.options = B.Options.from_buffer_copy(options if options is not None else renderer.options)
        T0 = np.stack([np.asarray(c["T_cw"], np.float32).reshape(12) for c in cameras])
        self.T0 = torch.from_numpy(T0).to(dev)
        self.T = self.T0.clone()
        self.m = torch.zeros((self.V, 6), device=dev)
        self.v = torch.zeros((self.V, 6), device=dev)
        self.step = torch.zeros(self.V, dtype=torch.int32, device=dev)
        self.target = target_rgb.contiguous()
        self.weight = weight.contiguous() if weight is not None else None
        self.out = renderer.empty_outputs(cameras, which=("rgb",))
        self.d_twist = torch.zeros((self.V, 6), device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.cam_arr = B.make_cameras(self.cameras)
        self.graph = None

    def reset(self):
        self.T.copy_(self.T0)
        self.m.zero_()
        self.v.zero_()
        self.step.zero_()

    def iteration(self):
        R, p = self.R, self.params
        g = B.make_gaussians(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["colors"],
                             p["sh_degree"])
        B.s3gs_render_fwd(R.ctx, R.state, g, self.cam_arr, self.V, self.T, self.options, self.out["rgb"], None,
                          None, None)
        # weighted L1 photometric loss fused into the pose-only backward
        B.s3gs_render_bwd_l1(R.ctx, R.state, self.out["rgb"], None, None, self.target, None, None, self.weight,
                             1.0, 0.0, 0.0, self.loss, None, None, None, None, None, self.d_twist, 0)
        B.s3gs_pose_update(R.ctx, self.V, self.d_twist, self.hp, self.m, self.v, self.step, self.T)

    def run_eager(self, iters=None):
        self.reset()
        for _ in range(self.iters if iters is None else iters):
            self.iteration()

    def capture(self, headroom: float = 1.5):
        """Size the state with an eager run, then record reset + iterations."""
        self.run_eager(1)
        torch.cuda.synchronize(self.R.device)
        _, K, _ = B.s3gs_state_check(self.R.ctx, self.R.state)
        P = sum(c["width"] * c["height"] for c in self.cameras)
        tiles = sum(((c["width"] + 7) // 8) * ((c["height"] + 7) // 8) for c in self.cameras)
        B.s3gs_reserve(self.R.ctx, self.R.state, int(self.params["means"].shape[0]), self.V, P, tiles,
                       int(K * headroom) + 4096)
        self.options.auto_grow = 0
        side = torch.cuda.Stream(device=self.R.device)
        side.wait_stream(torch.cuda.current_stream(self.R.device))
        with torch.cuda.stream(side):
            self.run_eager(1)
        torch.cuda.current_stream(self.R.device).wait_stream(side)
        torch.cuda.synchronize(self.R.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.reset()
            for _ in range(self.iters):
                self.iteration()
        torch.cuda.synchronize(self.R.device)
        return self.graph

    def run(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def check(self):
        """Raises if a replay overflowed the reserved duplicate capacity."""
        B.s3gs_state_check(self.R.ctx, self.R.state)

    def poses(self):
        return self.T.view(self.V, 3, 4).cpu().numpy()


class MapOptimizer:
    """One mapping iteration of the keyframe window (Eq. 17), entirely on the
    device: batched render of every window view, the mapping loss
    alpha L_pho + (1 - alpha) L_geo (+ an optional depth term) against the
    views' images and aligned pointmaps, the backward to all Gaussian
    parameters and the window twists, the fused Adam step with L_iso (Eq. 16)
    and the pose step with retraction. ``capture()`` records ``iters``
    iterations into one CUDA graph."""

    def __init__(self, renderer, params: dict, cameras, t_rgb, t_pointmap=None, t_depth=None, alpha=0.98,
                 w_depth=0.0, hp: B.MapAdam | None = None, pose_hp: B.PoseAdam | None = None, frozen=None,
                 iters: int = 1, options: B.Options | None = None):
        import numpy as np
        self.R = renderer
        self.p = params
        self.cameras = [dict(c) for c in cameras]
        self.V = len(cameras)
        dev = renderer.device
        self.hp = hp if hp is not None else B.s3gs_map_adam_default()
        self.pose_hp = pose_hp if pose_hp is not None else B.s3gs_pose_adam_default()
        self.iters = int(iters)
        self.options = B.Options.from_buffer_copy(options if options is not None else renderer.options)
        self.alpha, self.w_depth = float(alpha), float(w_depth)
        self.t_rgb, self.t_pm, self.t_depth = t_rgb, t_pointmap, t_depth
        T0 = np.stack([np.asarray(c["T_cw"], np.float32).reshape(12) for c in cameras])
        self.T = torch.from_numpy(T0).to(dev)
        self.frozen = frozen
        self.m = {k: torch.zeros_like(params[k]) for k in B.MAP_TENSORS}
        self.v = {k: torch.zeros_like(params[k]) for k in B.MAP_TENSORS}
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.pm_ = torch.zeros((self.V, 6), device=dev)
        self.pv_ = torch.zeros((self.V, 6), device=dev)
        self.pstep = torch.zeros(self.V, dtype=torch.int32, device=dev)
        self.out = renderer.empty_outputs(cameras)
        self.grads = {k: torch.zeros_like(params[k]) for k in B.MAP_TENSORS}
        self.d_twist = torch.zeros((self.V, 6), device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.cam_arr = B.make_cameras(self.cameras)
        self.graph = None

    def iteration(self):
        R, p, g = self.R, self.p, self.grads
        gs = B.make_gaussians(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["colors"],
                              p["sh_degree"])
        B.s3gs_render_fwd(R.ctx, R.state, gs, self.cam_arr, self.V, self.T, self.options, self.out["rgb"],
                          self.out["depth"], self.out["pointmap"], None)
        # mapping loss (Eq. 17) fused into the backward
        B.s3gs_render_bwd_l1(R.ctx, R.state, self.out["rgb"], self.out["depth"], self.out["pointmap"], self.t_rgb,
                             self.t_depth, self.t_pm, None, self.alpha,
                             self.w_depth if self.t_depth is not None else 0.0,
                             (1.0 - self.alpha) if self.t_pm is not None else 0.0, self.loss,
                             g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["colors"], self.d_twist, 0)
        B.s3gs_map_adam_step(R.ctx, p, g, self.m, self.v, self.step, self.hp)
        B.s3gs_pose_update(R.ctx, self.V, self.d_twist, self.pose_hp, self.pm_, self.pv_, self.pstep, self.T,
                           None, self.frozen)

    def capture(self, headroom: float = 1.5):
        """Size the state with one eager iteration, then record ``iters`` iterations.
        The eager iteration is a real step; call it part of the optimisation."""
        self.iteration()
        torch.cuda.synchronize(self.R.device)
        _, K, _ = B.s3gs_state_check(self.R.ctx, self.R.state)
        P = sum(c["width"] * c["height"] for c in self.cameras)
        tiles = sum(((c["width"] + 7) // 8) * ((c["height"] + 7) // 8) for c in self.cameras)
        B.s3gs_reserve(self.R.ctx, self.R.state, int(self.p["means"].shape[0]), self.V, P, tiles,
                       int(K * headroom) + 4096)
        self.options.auto_grow = 0
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device=self.R.device)
        side.wait_stream(torch.cuda.current_stream(self.R.device))
        with torch.cuda.graph(self.graph, stream=side):
            for _ in range(self.iters):
                self.iteration()
        torch.cuda.synchronize(self.R.device)
        return self.graph

    def run(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def check(self):
        B.s3gs_state_check(self.R.ctx, self.R.state)
