"""ctypes binding of ``libs3gs.so`` (C ABI in ``include/s3gs.h``).

Argument marshalling only: every computation runs in the CUDA library. The
functions keep the C names; tensors are passed as device pointers and the
current torch CUDA stream is used unless one is given. There is no fallback:
if the library is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

__all__ = [
    "S3GS_OK", "S3GS_E_INVALID", "S3GS_E_CAPACITY", "S3GS_E_CUDA", "S3GS_E_TIMEOUT",
    "S3GS_E_NOMEM", "S3GS_E_STATE", "S3GS_MAX_VIEWS", "S3GSError", "Gaussians", "Camera",
    "Options", "lib", "s3gs_options_default", "s3gs_create", "s3gs_destroy", "s3gs_last_error",
    "s3gs_state_create", "s3gs_state_destroy", "s3gs_reserve", "s3gs_render_fwd",
    "s3gs_render_bwd", "s3gs_render_bwd_l1", "s3gs_state_check", "s3gs_mapping_loss", "s3gs_debug_records",
    "s3gs_debug_binning", "s3gs_debug_cover", "s3gs_set_counting", "s3gs_read_counters", "s3gs_version",
    "s3gs_set_timing", "s3gs_read_timing", "STAGES", "s3gs_mapping_loss_noalloc",
    "make_cameras", "make_gaussians", "check", "AlignParams", "s3gs_align_params_default",
    "s3gs_scale_align_workspace", "s3gs_scale_align", "s3gs_pointmap_replace", "s3gs_scale_remedy", "view_sizes",
    "PoseAdam", "s3gs_pose_adam_default", "s3gs_se3_exp", "s3gs_pose_update", "KeyframeParams",
    "s3gs_covisibility", "s3gs_median_depth_workspace", "s3gs_median_depth", "s3gs_keyframe_params_default",
    "s3gs_keyframe_is_new", "s3gs_keyframe_window_update", "MapAdam", "s3gs_map_adam_default",
    "s3gs_map_adam_step", "MAP_TENSORS",
]

S3GS_OK, S3GS_E_INVALID, S3GS_E_CAPACITY, S3GS_E_CUDA = 0, -1, -2, -3
S3GS_E_TIMEOUT, S3GS_E_NOMEM, S3GS_E_STATE = -4, -5, -6
S3GS_MAX_VIEWS = 32
_NAMES = {0: "OK", -1: "INVALID", -2: "CAPACITY", -3: "CUDA", -4: "TIMEOUT", -5: "NOMEM", -6: "STATE"}


class S3GSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"s3gs {_NAMES.get(status, status)}: {msg}")
        self.status = status


class Gaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity_logits", ctypes.c_void_p),
                ("colors", ctypes.c_void_p)]


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("T_cw", ctypes.c_float * 12)]


class Options(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("pixels_per_thread", ctypes.c_int32), ("bwd_pixels_per_thread", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("recompute", ctypes.c_int32),
                ("auto_grow", ctypes.c_int32), ("near_z", ctypes.c_float), ("guard_slope", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("full_lists", ctypes.c_int32)]


class AlignParams(ctypes.Structure):
    _fields_ = [("patch", ctypes.c_int32), ("delta_mu", ctypes.c_float), ("delta_sigma", ctypes.c_float),
                ("eps_r", ctypes.c_float), ("max_iter", ctypes.c_int32), ("tau", ctypes.c_float)]


class KeyframeParams(ctypes.Structure):
    _fields_ = [("k_iou", ctypes.c_float), ("k_d", ctypes.c_float), ("k_oc", ctypes.c_float),
                ("max_window", ctypes.c_int32)]


class MapAdam(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("lr_means", "lr_log_scales", "lr_quats", "lr_opacity", "lr_colors",
                                              "lr_colors_rest", "beta1", "beta2", "eps", "lambda_iso")]


class PoseAdam(ctypes.Structure):
    _fields_ = [("lr_rho", ctypes.c_float), ("lr_phi", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


_P = ctypes.c_void_p
_lib = None


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libs3gs.so is not built ({path}); run __graft_entry__.build() or "
                          "python -m paper_2507_03737_gb300.build")
    L = ctypes.CDLL(path)
    sig = {
        "s3gs_options_default": (None, [ctypes.POINTER(Options)]),
        "s3gs_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P)]),
        "s3gs_destroy": (None, [_P]),
        "s3gs_last_error": (ctypes.c_char_p, [_P]),
        "s3gs_state_create": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
        "s3gs_state_destroy": (None, [_P]),
        "s3gs_reserve": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int64]),
        "s3gs_render_fwd": (ctypes.c_int, [_P, _P, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera),
                                           ctypes.c_int32, _P, ctypes.POINTER(Options), _P, _P, _P, _P, _P]),
        "s3gs_render_bwd": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                           ctypes.c_int32, _P]),
        "s3gs_render_bwd_l1": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float,
                                              ctypes.c_float, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]),
        "s3gs_state_check": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64)]),
        "s3gs_mapping_loss": (ctypes.c_int, [_P, ctypes.POINTER(Camera), ctypes.c_int32, _P, _P, _P, _P, _P,
                                             _P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                             _P, _P, _P, _P, _P]),
        "s3gs_debug_records": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P]),
        "s3gs_debug_cover": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
        "s3gs_debug_binning": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int64)]),
        "s3gs_set_counting": (ctypes.c_int, [_P, ctypes.c_int32]),
        "s3gs_read_counters": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "s3gs_mapping_loss_noalloc": (ctypes.c_int, [ctypes.POINTER(Camera), ctypes.c_int32, _P, _P, _P, _P, _P,
                                                     _P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                                     _P, _P, _P, _P, _P, ctypes.c_char_p, ctypes.c_size_t]),
        "s3gs_set_timing": (ctypes.c_int, [_P, ctypes.c_int32]),
        "s3gs_read_timing": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
        "s3gs_version": (ctypes.c_char_p, []),
        "s3gs_align_params_default": (None, [ctypes.POINTER(AlignParams)]),
        "s3gs_scale_align_workspace": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32,
                                                      ctypes.POINTER(ctypes.c_size_t)]),
        "s3gs_scale_align": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, ctypes.POINTER(AlignParams), _P, _P,
                                            _P, _P, _P, _P, ctypes.c_size_t, _P]),
        "s3gs_pointmap_replace": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, _P, ctypes.c_float, _P, _P, _P,
                                                 _P, _P]),
        "s3gs_scale_remedy": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.c_int64, _P,
                                             _P, _P]),
        "s3gs_covisibility": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
        "s3gs_median_depth_workspace": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
        "s3gs_median_depth": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_size_t, _P]),
        "s3gs_keyframe_params_default": (None, [ctypes.POINTER(KeyframeParams)]),
        "s3gs_keyframe_is_new": (ctypes.c_int32, [ctypes.POINTER(KeyframeParams), ctypes.c_float, ctypes.c_float,
                                                  ctypes.c_float]),
        "s3gs_keyframe_window_update": (ctypes.c_int, [ctypes.POINTER(KeyframeParams), _P, _P, ctypes.c_int32,
                                                       ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_int32)]),
        "s3gs_map_adam_default": (None, [ctypes.POINTER(MapAdam)]),
        "s3gs_map_adam_step": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P, _P,
                                              ctypes.POINTER(MapAdam), _P]),
        "s3gs_pose_adam_default": (None, [ctypes.POINTER(PoseAdam)]),
        "s3gs_se3_exp": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P]),
        "s3gs_pose_update": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.POINTER(PoseAdam), _P, _P, _P, _P, _P,
                                            _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or t.dtype not in (torch.float32, torch.int32, torch.uint32, torch.int64, torch.uint8):
        raise TypeError("expected a float32 / int32 / int64 / uint8 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def check(ctx, status):
    if status != S3GS_OK:
        msg = lib().s3gs_last_error(ctx).decode() if ctx else ""
        raise S3GSError(status, msg)


def s3gs_version() -> str:
    return lib().s3gs_version().decode()


def s3gs_options_default(**kw) -> Options:
    o = Options()
    lib().s3gs_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "bg":
            for i in range(3):
                o.bg[i] = float(v[i])
        else:
            setattr(o, k, v)
    return o


def s3gs_create(device: int = 0):
    h = _P()
    st = lib().s3gs_create(int(device), ctypes.byref(h))
    if st != S3GS_OK:
        raise S3GSError(st, f"cannot create a context on device {device}")
    return h.value


def s3gs_destroy(ctx):
    lib().s3gs_destroy(ctx)


def s3gs_last_error(ctx) -> str:
    return lib().s3gs_last_error(ctx).decode()


def s3gs_state_create(ctx):
    h = _P()
    check(ctx, lib().s3gs_state_create(ctx, ctypes.byref(h)))
    return h.value


def s3gs_state_destroy(state):
    lib().s3gs_state_destroy(state)


def s3gs_reserve(ctx, state, n, n_views, total_pixels, total_tiles, max_duplicates):
    check(ctx, lib().s3gs_reserve(ctx, state, int(n), int(n_views), int(total_pixels),
                                  int(total_tiles), int(max_duplicates)))


def make_gaussians(means, log_scales, quats, opacity_logits, colors, sh_degree) -> Gaussians:
    n = int(means.shape[0])
    return Gaussians(n, int(sh_degree), _ptr(means), _ptr(log_scales), _ptr(quats),
                     _ptr(opacity_logits), _ptr(colors))


def make_cameras(cameras):
    """cameras: list of dicts (width, height, fx, fy, cx, cy, T_cw 3x4)."""
    arr = (Camera * len(cameras))()
    for k, c in enumerate(cameras):
        arr[k].width, arr[k].height = int(c["width"]), int(c["height"])
        arr[k].fx, arr[k].fy, arr[k].cx, arr[k].cy = (float(c["fx"]), float(c["fy"]),
                                                       float(c["cx"]), float(c["cy"]))
        T = [float(x) for x in __import__("numpy").asarray(c["T_cw"], dtype="float64").reshape(12)]
        for i in range(12):
            arr[k].T_cw[i] = T[i]
    return arr


def s3gs_render_fwd(ctx, state, gaussians: Gaussians, cams, n_views, T_cw_device, options: Options,
                    rgb, depth, pointmap, alpha, stream=None):
    check(ctx, lib().s3gs_render_fwd(ctx, state, ctypes.byref(gaussians), cams, int(n_views),
                                     _ptr(T_cw_device), ctypes.byref(options), _ptr(rgb), _ptr(depth),
                                     _ptr(pointmap), _ptr(alpha), _stream(stream)))


def s3gs_render_bwd(ctx, state, d_rgb, d_depth, d_pointmap, d_alpha, d_means, d_log_scales, d_quats,
                    d_opacity_logits, d_colors, d_twist, accumulate=0, stream=None):
    check(ctx, lib().s3gs_render_bwd(ctx, state, _ptr(d_rgb), _ptr(d_depth), _ptr(d_pointmap),
                                     _ptr(d_alpha), _ptr(d_means), _ptr(d_log_scales), _ptr(d_quats),
                                     _ptr(d_opacity_logits), _ptr(d_colors), _ptr(d_twist),
                                     int(accumulate), _stream(stream)))


def s3gs_render_bwd_l1(ctx, state, rgb, depth, pointmap, t_rgb, t_depth, t_pointmap, mask, w_rgb, w_depth, w_geo,
                       loss_device, d_means, d_log_scales, d_quats, d_opacity_logits, d_colors, d_twist, accumulate=0,
                       stream=None):
    check(ctx, lib().s3gs_render_bwd_l1(ctx, state, _ptr(rgb), _ptr(depth), _ptr(pointmap), _ptr(t_rgb),
                                        _ptr(t_depth), _ptr(t_pointmap), _ptr(mask), float(w_rgb), float(w_depth),
                                        float(w_geo), _ptr(loss_device), _ptr(d_means), _ptr(d_log_scales),
                                        _ptr(d_quats), _ptr(d_opacity_logits), _ptr(d_colors), _ptr(d_twist),
                                        int(accumulate), _stream(stream)))


def s3gs_state_check(ctx, state, raise_on_error=True):
    k = ctypes.c_int64(); cap = ctypes.c_int64()
    st = lib().s3gs_state_check(ctx, state, ctypes.byref(k), ctypes.byref(cap))
    if raise_on_error:
        check(ctx, st)
    return st, k.value, cap.value


def s3gs_mapping_loss(ctx, cams, n_views, rgb, depth, pointmap, t_rgb, t_depth, t_pointmap, mask,
                      w_rgb, w_depth, w_geo, d_rgb, d_depth, d_pointmap, loss_device, stream=None):
    check(ctx, lib().s3gs_mapping_loss(ctx, cams, int(n_views), _ptr(rgb), _ptr(depth), _ptr(pointmap),
                                       _ptr(t_rgb), _ptr(t_depth), _ptr(t_pointmap), _ptr(mask),
                                       float(w_rgb), float(w_depth), float(w_geo), _ptr(d_rgb),
                                       _ptr(d_depth), _ptr(d_pointmap), _ptr(loss_device),
                                       _stream(stream)))


def s3gs_mapping_loss_noalloc(cams, n_views, rgb, depth, pointmap, t_rgb, t_depth, t_pointmap, mask,
                              w_rgb, w_depth, w_geo, d_rgb, d_depth, d_pointmap, loss_device, stream=None):
    """Allocation-free mapping loss (no context); raises S3GSError with the library's message."""
    buf = ctypes.create_string_buffer(256)
    st = lib().s3gs_mapping_loss_noalloc(cams, int(n_views), _ptr(rgb), _ptr(depth), _ptr(pointmap), _ptr(t_rgb),
                                         _ptr(t_depth), _ptr(t_pointmap), _ptr(mask), float(w_rgb), float(w_depth),
                                         float(w_geo), _ptr(d_rgb), _ptr(d_depth), _ptr(d_pointmap),
                                         _ptr(loss_device), _stream(stream), buf, len(buf))
    if st != S3GS_OK:
        raise S3GSError(st, buf.value.decode())


def s3gs_debug_records(ctx, state, n_records):
    import numpy as np
    xy = np.zeros((n_records, 2), np.float32); co = np.zeros((n_records, 4), np.float32)
    rz = np.zeros((n_records, 4), np.float32); ext = np.zeros((n_records, 2), np.int32)
    check(ctx, lib().s3gs_debug_records(ctx, state, int(n_records), xy.ctypes.data, co.ctypes.data,
                                        rz.ctypes.data, ext.ctypes.data))
    return dict(xy=xy, conic_opacity=co, rgb_depth=rz, extent=ext)


def s3gs_debug_cover(ctx, state, n_records):
    import numpy as np
    q = np.zeros(n_records, np.float32)
    check(ctx, lib().s3gs_debug_cover(ctx, state, int(n_records), q.ctypes.data))
    return q


def s3gs_debug_binning(ctx, state):
    import numpy as np
    nt = ctypes.c_int64(); nk = ctypes.c_int64()
    check(ctx, lib().s3gs_debug_binning(ctx, state, None, None, None, ctypes.byref(nt), ctypes.byref(nk)))
    keys = np.zeros(max(nk.value, 1), np.uint64); vals = np.zeros(max(nk.value, 1), np.uint32)
    ranges = np.zeros(nt.value + 1, np.int64)
    check(ctx, lib().s3gs_debug_binning(ctx, state, keys.ctypes.data, vals.ctypes.data, ranges.ctypes.data,
                                        ctypes.byref(nt), ctypes.byref(nk)))
    return keys[:nk.value], vals[:nk.value], ranges


STAGES = ("project", "scan", "emit", "tile_sort", "tile_order", "blend_fwd", "blend_bwd", "det_reduce",
          "project_bwd", "twist_reduce", "loss")


def s3gs_set_timing(ctx, enable: bool):
    check(ctx, lib().s3gs_set_timing(ctx, int(bool(enable))))


def s3gs_read_timing(ctx) -> dict:
    arr = (ctypes.c_float * len(STAGES))()
    check(ctx, lib().s3gs_read_timing(ctx, arr, len(STAGES)))
    return {k: float(arr[i]) for i, k in enumerate(STAGES) if arr[i] >= 0}


def s3gs_set_counting(ctx, enable: bool):
    check(ctx, lib().s3gs_set_counting(ctx, int(bool(enable))))


def s3gs_read_counters(ctx, state):
    a = ctypes.c_int64(); b = ctypes.c_int64(); c = ctypes.c_int64()
    check(ctx, lib().s3gs_read_counters(ctx, state, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return dict(fwd_processed=a.value, fwd_blended=b.value, bwd_processed=c.value)


def view_sizes(cameras_or_wh):
    """Host int32 [n_views][2] (width, height) array from camera dicts or (w, h) pairs."""
    wh = []
    for c in cameras_or_wh:
        wh += [int(c["width"]), int(c["height"])] if isinstance(c, dict) else [int(c[0]), int(c[1])]
    arr = (ctypes.c_int32 * len(wh))(*wh)
    return arr, len(wh) // 2


def s3gs_align_params_default(**kw) -> AlignParams:
    p = AlignParams()
    lib().s3gs_align_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def s3gs_scale_align_workspace(view_wh, n_views, patch) -> int:
    b = ctypes.c_size_t()
    st = lib().s3gs_scale_align_workspace(view_wh, int(n_views), int(patch), ctypes.byref(b))
    if st != S3GS_OK:
        raise S3GSError(st, "scale_align_workspace: sizes out of range")
    return b.value


def s3gs_scale_align(ctx, view_wh, n_views, X_r, X_p, params, sigma_init, sigma, n_cp, insufficient, cp_mask,
                     workspace, stream=None):
    ws = workspace.numel() * workspace.element_size()
    check(ctx, lib().s3gs_scale_align(ctx, view_wh, int(n_views), _ptr(X_r), _ptr(X_p), ctypes.byref(params),
                                      _ptr(sigma_init), _ptr(sigma), _ptr(n_cp), _ptr(insufficient), _ptr(cp_mask),
                                      workspace.data_ptr(), ws, _stream(stream)))


def s3gs_pointmap_replace(ctx, view_wh, n_views, X_r, X_p, sigma, eps_m, X_r_hat, X_p_hat, replaced, n_replaced,
                          stream=None):
    check(ctx, lib().s3gs_pointmap_replace(ctx, view_wh, int(n_views), _ptr(X_r), _ptr(X_p), _ptr(sigma),
                                           float(eps_m), _ptr(X_r_hat), _ptr(X_p_hat), _ptr(replaced),
                                           _ptr(n_replaced), _stream(stream)))


def s3gs_scale_remedy(ctx, X_ak_hat, hw_ak, X_n, hw_n, matches, n_matches, sigma, n_used, stream=None):
    check(ctx, lib().s3gs_scale_remedy(ctx, _ptr(X_ak_hat), int(hw_ak), _ptr(X_n), int(hw_n), _ptr(matches),
                                       int(n_matches), _ptr(sigma), _ptr(n_used), _stream(stream)))


def s3gs_pose_adam_default(**kw) -> PoseAdam:
    p = PoseAdam()
    lib().s3gs_pose_adam_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def s3gs_se3_exp(ctx, n, tau, E, stream=None):
    check(ctx, lib().s3gs_se3_exp(ctx, int(n), _ptr(tau), _ptr(E), _stream(stream)))


def s3gs_pose_update(ctx, n_views, d_twist, hp, adam_m, adam_v, step, T_cw, delta=None, frozen=None, stream=None):
    check(ctx, lib().s3gs_pose_update(ctx, int(n_views), _ptr(d_twist), ctypes.byref(hp), _ptr(adam_m), _ptr(adam_v),
                                      _ptr(step), _ptr(T_cw), _ptr(delta), _ptr(frozen), _stream(stream)))


def s3gs_covisibility(ctx, state, counts, iou=None, oc=None, stream=None):
    check(ctx, lib().s3gs_covisibility(ctx, state, _ptr(counts), _ptr(iou), _ptr(oc), _stream(stream)))


def s3gs_median_depth_workspace(n_views) -> int:
    b = ctypes.c_size_t()
    st = lib().s3gs_median_depth_workspace(int(n_views), ctypes.byref(b))
    if st != S3GS_OK:
        raise S3GSError(st, "median_depth_workspace: n_views out of range")
    return b.value


def s3gs_median_depth(ctx, view_wh, n_views, depth, median, n_valid, workspace, stream=None):
    ws = workspace.numel() * workspace.element_size()
    check(ctx, lib().s3gs_median_depth(ctx, view_wh, int(n_views), _ptr(depth), _ptr(median), _ptr(n_valid),
                                       workspace.data_ptr(), ws, _stream(stream)))


def s3gs_keyframe_params_default(**kw) -> KeyframeParams:
    p = KeyframeParams()
    lib().s3gs_keyframe_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def s3gs_keyframe_is_new(params, iou_ij, d_ij, median_depth_i) -> bool:
    r = lib().s3gs_keyframe_is_new(ctypes.byref(params), float(iou_ij), float(d_ij), float(median_depth_i))
    if r < 0:
        raise S3GSError(S3GS_E_INVALID, "keyframe_is_new: NULL parameters")
    return bool(r)


def s3gs_keyframe_window_update(params, window_ids, oc_with_new, new_id):
    n = len(window_ids)
    ids = (ctypes.c_int32 * max(n, 1))(*[int(x) for x in window_ids])
    oc = (ctypes.c_float * max(n, 1))(*[float(x) for x in oc_with_new])
    out = (ctypes.c_int32 * (n + 1))()
    m = ctypes.c_int32()
    st = lib().s3gs_keyframe_window_update(ctypes.byref(params), ids, oc, n, int(new_id), out, ctypes.byref(m))
    if st != S3GS_OK:
        raise S3GSError(st, "keyframe_window_update: bad arguments")
    return [int(out[k]) for k in range(m.value)]


MAP_TENSORS = ("means", "log_scales", "quats", "opacity_logits", "colors")


def s3gs_map_adam_default(**kw) -> MapAdam:
    p = MapAdam()
    lib().s3gs_map_adam_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def s3gs_map_adam_step(ctx, params: dict, grads: dict, m: dict, v: dict, step, hp, stream=None):
    """params / grads / m / v: dicts of CUDA tensors keyed by MAP_TENSORS (a missing
    gradient is zero); params["sh_degree"] gives the colour layout."""
    arr = lambda d, req: (_P * 5)(*[_ptr(d.get(k)) if not req else _ptr(d[k]) for k in MAP_TENSORS])
    n = int(params["means"].shape[0])
    check(ctx, lib().s3gs_map_adam_step(ctx, n, int(params["sh_degree"]), arr(params, True), arr(grads, False),
                                        arr(m, True), arr(v, True), _ptr(step), ctypes.byref(hp), _stream(stream)))
