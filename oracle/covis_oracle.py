"""Oracle of keyframe covisibility and window management (supplementary
material, "Keyframe Management", Eq. S1/S2 and the rules after them).
Test infrastructure only; plain numpy / Python.

Readings taken where the text leaves the computation open:
  * The visible set G_i^v of view i is the set of Gaussians the rasteriser
    projects into view i with a non-empty pixel footprint (the renderer's
    per-record visibility); ``projected_sets`` gives the FP64 version of that
    rule (mean in front of the near plane and inside the guard cone,
    3-sigma bounding box meeting the pixel grid) and ``sets_from_extents``
    the exact set of a render from its per-record integer extents.
  * IOU and OC are 0 when their denominator is 0.
  * The median depth of a frame is the element of rank floor((N - 1) / 2) of
    the sorted depths of its N pixels with depth > 0 (the lower median), 0 if
    N = 0.
  * Window update after a new keyframe joins: every window keyframe whose OC
    with the new one is below k_o leaves; then, while the window (the new
    keyframe included) is larger than its maximum size, the remaining
    keyframe with the lowest OC leaves (the earlier one on ties). The new
    keyframe is appended last and never removed; the order of the others is
    kept.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

__all__ = ["projected_sets", "sets_from_extents", "counts", "iou_oc", "median_depth", "is_new_keyframe",
           "window_update", "DEFAULTS"]

DEFAULTS = dict(k_iou=0.9, k_d=0.08, k_oc=0.3, max_window=8)


def projected_sets(scene, cameras, near_z=0.2):
    """Boolean [V][n] visibility from the FP64 projection (guard slope 1.5), and
    the distance (in pixels) of each footprint's edge from the image border
    (0 where the near-plane or guard decision itself is within 1e-5 of its
    threshold; small = ambiguous)."""
    V, n = len(cameras), scene.n
    vis = np.zeros((V, n), dtype=bool)
    slack = np.full((V, n), np.inf)
    for v, cam in enumerate(cameras):
        p = O.project(scene, cam, near_z)
        ok = p["valid"] > 0
        rx = 3.0 * np.sqrt(np.maximum(p["cov_a"], 0.0))
        ry = 3.0 * np.sqrt(np.maximum(p["cov_c"], 0.0))
        W, H = cam["width"], cam["height"]
        # footprint [u - rx, u + rx] x [v - ry, v + ry] meets [0, W - 1] x [0, H - 1]
        gx = np.minimum(p["u"] + rx, (W - 1) - (p["u"] - rx))
        gy = np.minimum(p["v"] + ry, (H - 1) - (p["v"] - ry))
        vis[v] = ok & (gx >= 0) & (gy >= 0)
        slack[v] = np.where(ok, np.minimum(np.abs(gx), np.abs(gy)), np.inf)
        # near-plane and guard-cone decisions within 1e-5 of their threshold are
        # ambiguous in FP32 as well
        T = np.asarray(cam["T_cw"], dtype=np.float64).reshape(3, 4)
        pc = np.asarray(scene.means, dtype=np.float64) @ T[:, :3].T + T[:, 3]
        z = pc[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            m = np.minimum(np.abs(z - near_z) / near_z,
                           np.minimum(np.abs(np.abs(pc[:, 0] / z) - 1.5), np.abs(np.abs(pc[:, 1] / z) - 1.5)) / 1.5)
        slack[v] = np.where((z > 0) & (m < 1e-5), 0.0, slack[v])
    return vis, slack


def sets_from_extents(extent, n_views):
    """Visibility [V][n] from per-record integer extents (rx > 0 = projected
    with a non-empty footprint), records ordered r = v * n + g."""
    e = np.asarray(extent).reshape(n_views, -1, 2)
    return e[:, :, 0] > 0


def counts(vis):
    """C[i][j] = |G_i & G_j| (C[i][i] = |G_i|)."""
    vis = np.asarray(vis, dtype=bool)
    V = vis.shape[0]
    C = np.zeros((V, V), dtype=np.int64)
    for i in range(V):
        for j in range(V):
            C[i, j] = int(np.count_nonzero(vis[i] & vis[j]))
    return C


def iou_oc(C):
    """Eq. S1 (IOU) and Eq. S2 (OC) from the intersection counts."""
    C = np.asarray(C, dtype=np.int64)
    V = C.shape[0]
    iou = np.zeros((V, V)); oc = np.zeros((V, V))
    for i in range(V):
        for j in range(V):
            union = C[i, i] + C[j, j] - C[i, j]
            small = min(C[i, i], C[j, j])
            iou[i, j] = C[i, j] / union if union > 0 else 0.0
            oc[i, j] = C[i, j] / small if small > 0 else 0.0
    return iou, oc


def median_depth(depth):
    """Lower median of the positive entries of one view's depth map."""
    d = np.asarray(depth).reshape(-1)
    valid = np.sort(d[d > 0])
    if valid.size == 0:
        return 0.0, 0
    return float(valid[(valid.size - 1) // 2]), int(valid.size)


def is_new_keyframe(iou_ij, d_ij, median_depth_i, k_iou=0.9, k_d=0.08):
    """Frame i joins the window when IOU(i, j) < k_I or d_ij > k_d * D_i."""
    return bool(iou_ij < k_iou or d_ij > k_d * median_depth_i)


def window_update(window_ids, oc_with_new, new_id, k_oc=0.3, max_window=8):
    keep = [(k, w, o) for k, (w, o) in enumerate(zip(window_ids, oc_with_new)) if not (o < k_oc)]
    while len(keep) + 1 > max_window and keep:
        worst = min(range(len(keep)), key=lambda t: (keep[t][2], keep[t][0]))
        keep.pop(worst)
    return [w for (_, w, _) in keep] + [new_id]
