"""ctypes front end of the FP64 oracle in ``s3gs_oracle.c`` (test infrastructure only).

The C file follows Sec. 3.1 (Eq. 1-2), Sec. 3.2.1 (Eq. 3-5) and Sec. 3.2.2
(Eq. 11) of the paper with no tiling; see its header for the readings it makes.
Inputs are the float32 scene arrays, widened exactly to float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = ["build_oracle", "lib", "cam_rows", "project", "render_fwd", "render_bwd",
           "bin_referee", "sh_real", "quat_to_rotmat", "num_threads", "set_num_threads", "set_guard",
           "pixel_offsets"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "s3gs_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U64 = ctypes.POINTER(ctypes.c_uint64)
_U32 = ctypes.POINTER(ctypes.c_uint32)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math, no FP contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            L = ctypes.CDLL(_SO)
            L.or_quat_to_rotmat.argtypes = [_D, _D]
            L.or_sh_real.argtypes = [ctypes.c_int, ctypes.c_int, _D]
            L.or_sh_real.restype = ctypes.c_double
            L.or_project.argtypes = [ctypes.c_int64, ctypes.c_int, _D, _D, _D, _D, _D, _D,
                                     ctypes.c_double, _D]
            L.or_render_fwd.argtypes = [ctypes.c_int64, ctypes.c_int, _D, _D, _D, _D, _D,
                                        ctypes.c_int, _D, ctypes.c_double, _D,
                                        _D, _D, _D, _D, _D, _I64]
            L.or_render_bwd.argtypes = [ctypes.c_int64, ctypes.c_int, _D, _D, _D, _D, _D,
                                        ctypes.c_int, _D, ctypes.c_double, _D,
                                        _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
            L.or_bin_referee.argtypes = [ctypes.c_int64, ctypes.c_int, _I32, ctypes.c_int,
                                         ctypes.c_int, _F, _F, _I32, _I32, _F, _F, _F, _U64, _U32, _I64]
            L.or_bin_referee.restype = ctypes.c_int64
            L.or_num_threads.restype = ctypes.c_int
            L.or_set_guard.argtypes = [ctypes.c_double]
            L.or_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _p(a, t=_D):
    return a.ctypes.data_as(t) if a is not None else None


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def cam_rows(cameras) -> np.ndarray:
    rows = []
    for c in cameras:
        T = np.asarray(c["T_cw"], dtype=np.float64).reshape(12)
        rows.append([c["width"], c["height"], c["fx"], c["fy"], c["cx"], c["cy"], *T])
    return np.ascontiguousarray(np.array(rows, dtype=np.float64).reshape(len(cameras), 18))


def pixel_offsets(cameras):
    off = [0]
    for c in cameras:
        off.append(off[-1] + c["width"] * c["height"])
    return off


def set_guard(g: float) -> None:
    """Guard-cone slope G (a Gaussian with |x/z| or |y/z| > G is not projected);
    <= 0 disables the cone. Default 1.5, as in the library."""
    lib().or_set_guard(float(g))


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


def quat_to_rotmat(q) -> np.ndarray:
    q = _d(q)
    R = np.zeros(9)
    lib().or_quat_to_rotmat(_p(q), _p(R))
    return R.reshape(3, 3)


def sh_real(l: int, m: int, d) -> float:
    d = _d(d)
    return float(lib().or_sh_real(int(l), int(m), _p(d)))


def _scene_arrays(scene):
    return (_d(scene.means), _d(scene.log_scales), _d(scene.quats), _d(scene.opacity_logits),
            _d(scene.colors))


def project(scene, cam, near_z: float = 0.2) -> dict:
    """Per-Gaussian FP64 projection for one camera (diagnostics)."""
    m, ls, q, ol, c = _scene_arrays(scene)
    row = cam_rows([cam])[0].copy()
    out = np.zeros((scene.n, 13))
    rc = lib().or_project(scene.n, scene.sh_degree, _p(m), _p(ls), _p(q), _p(ol), _p(c), _p(row),
                          near_z, _p(out))
    assert rc == 0
    keys = ["valid", "u", "v", "A", "B", "C", "opacity", "depth", "r", "g", "b", "cov_a", "cov_c"]
    return {k: out[:, i] for i, k in enumerate(keys)}


def render_fwd(scene, cameras=None, near_z: float = 0.2, bg=None) -> dict:
    """FP64 render of all views. Returns packed planar outputs plus per-pixel margins."""
    cameras = scene.cameras if cameras is None else cameras
    m, ls, q, ol, c = _scene_arrays(scene)
    rows = cam_rows(cameras)
    P = pixel_offsets(cameras)[-1]
    rgb = np.zeros(3 * P); depth = np.zeros(P); pm = np.zeros(3 * P); alpha = np.zeros(P)
    margin = np.zeros(P); ncon = np.zeros(P, dtype=np.int64)
    bgv = _d(bg) if bg is not None else None
    rc = lib().or_render_fwd(scene.n, scene.sh_degree, _p(m), _p(ls), _p(q), _p(ol), _p(c),
                             len(cameras), _p(rows), near_z, _p(bgv), _p(rgb), _p(depth), _p(pm),
                             _p(alpha), _p(margin), _p(ncon, _I64))
    assert rc == 0
    return dict(rgb=rgb, depth=depth, pointmap=pm, alpha=alpha, margin=margin, n_contrib=ncon)


def render_bwd(scene, d_rgb=None, d_depth=None, d_pointmap=None, d_alpha=None, cameras=None,
               near_z: float = 0.2, bg=None) -> dict:
    """FP64 analytic gradients of sum(d_out * out) over the given upstream gradients."""
    cameras = scene.cameras if cameras is None else cameras
    m, ls, q, ol, c = _scene_arrays(scene)
    rows = cam_rows(cameras)
    n, V = scene.n, len(cameras)
    nc = (scene.sh_degree + 1) ** 2
    out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacity_logits=np.zeros(n), colors=np.zeros((n, nc, 3)), twist=np.zeros((V, 6)))
    bgv = _d(bg) if bg is not None else None
    args = [(_d(x) if x is not None else None) for x in (d_rgb, d_depth, d_pointmap, d_alpha)]
    rc = lib().or_render_bwd(n, scene.sh_degree, _p(m), _p(ls), _p(q), _p(ol), _p(c), V, _p(rows),
                             near_z, _p(bgv), *[_p(a) for a in args],
                             _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]),
                             _p(out["opacity_logits"]), _p(out["colors"]), _p(out["twist"]))
    assert rc == 0
    return out


def bin_referee(view_wh, tile_w, tile_h, u, v, rx, ry, z, conic=None, q_cover=None):
    """Integer referee: stable (tile, depth) keys, values and per-tile ranges.
    conic ([records][3] = A, B, C) and q_cover ([records]) enable the ellipse
    test of the tile cover; without them every tile of the rectangle is listed."""
    n_views = len(view_wh)
    wh = np.ascontiguousarray(np.asarray(view_wh, dtype=np.int32).reshape(n_views, 2))
    u = np.ascontiguousarray(u, dtype=np.float32); v = np.ascontiguousarray(v, dtype=np.float32)
    rx = np.ascontiguousarray(rx, dtype=np.int32); ry = np.ascontiguousarray(ry, dtype=np.int32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    cn = None if conic is None else np.ascontiguousarray(np.asarray(conic, dtype=np.float32).reshape(-1, 3))
    qc = None if q_cover is None else np.ascontiguousarray(q_cover, dtype=np.float32)
    n = u.size // n_views
    L = lib()
    K = L.or_bin_referee(n, n_views, _p(wh, _I32), tile_w, tile_h, _p(u, _F), _p(v, _F),
                         _p(rx, _I32), _p(ry, _I32), _p(z, _F), _p(cn, _F), _p(qc, _F), None, None, None)
    assert K >= 0
    n_tiles = sum(((w + tile_w - 1) // tile_w) * ((h + tile_h - 1) // tile_h) for w, h in wh)
    keys = np.zeros(max(K, 1), dtype=np.uint64); vals = np.zeros(max(K, 1), dtype=np.uint32)
    ranges = np.zeros(n_tiles + 1, dtype=np.int64)
    K2 = L.or_bin_referee(n, n_views, _p(wh, _I32), tile_w, tile_h, _p(u, _F), _p(v, _F),
                          _p(rx, _I32), _p(ry, _I32), _p(z, _F), _p(cn, _F), _p(qc, _F), _p(keys, _U64),
                          _p(vals, _U32), _p(ranges, _I64))
    assert K2 == K
    return keys[:K], vals[:K], ranges
