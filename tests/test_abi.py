"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point.

No compute call is made here (no GPU is needed).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
HEADERS = sorted(os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h"))


def declared_functions():
    names = []
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"\b(s3gs_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    from paper_2507_03737_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("s3gs_create", "s3gs_destroy", "s3gs_render_fwd", "s3gs_render_bwd", "s3gs_reserve",
                 "s3gs_state_create", "s3gs_state_check", "s3gs_mapping_loss", "s3gs_last_error",
                 "s3gs_scale_align", "s3gs_pointmap_replace", "s3gs_scale_remedy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.s3gs_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.s3gs_version()
    from paper_2507_03737_gb300 import binding as B
    o = B.s3gs_options_default()
    assert (o.tile_w, o.tile_h, o.auto_grow, o.full_lists) == (16, 16, 1, 0)
    assert abs(o.near_z - 0.2) < 1e-7
    # null arguments are rejected without touching the GPU
    assert lib.s3gs_create(0, None) == B.S3GS_E_INVALID


def test_binding_struct_layout_matches_header():
    from paper_2507_03737_gb300 import binding as B
    assert ctypes.sizeof(B.Camera) == 4 * (2 + 4 + 12)
    assert ctypes.sizeof(B.Options) == 4 * (9 + 2 + 3 + 1)
    assert B.Options.full_lists.offset == 4 * (9 + 2 + 3)
    assert B.Gaussians.means.offset == 16


def test_no_cpu_fallback_in_product_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2507_03737_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "s3gs_oracle" not in src, f


def test_align_params_and_workspace_are_host_only(lib):
    from paper_2507_03737_gb300 import binding as B
    assert ctypes.sizeof(B.AlignParams) == 4 * 6
    p = B.s3gs_align_params_default()
    assert (p.patch, p.max_iter) == (10, 3)
    assert abs(p.delta_mu - 0.3) < 1e-7 and abs(p.delta_sigma - 0.3) < 1e-7
    assert abs(p.eps_r - 0.1) < 1e-7 and abs(p.tau - 0.01) < 1e-9
    wh, nv = B.view_sizes([(1241, 376), (23, 7)])
    # 1241x376 at P = 10: 38 patch rows x ceil(125 / 12) CTAs (12 patches of a 128-thread CTA);
    # 23x7: 1 x 1; 16 bytes per CTA
    assert B.s3gs_scale_align_workspace(wh, nv, 10) == 16 * (38 * 11 + 1)
    for bad in (0, 33):
        with pytest.raises(B.S3GSError):
            B.s3gs_scale_align_workspace(wh, nv, bad)


def test_keyframe_window_logic_matches_oracle(lib):
    """Host-only keyframe rules of the library against the oracle's reading."""
    import numpy as np
    from oracle import covis_oracle as C
    from paper_2507_03737_gb300 import binding as B
    p = B.s3gs_keyframe_params_default()
    assert (abs(p.k_iou - 0.9) < 1e-7, abs(p.k_d - 0.08) < 1e-7, abs(p.k_oc - 0.3) < 1e-7, p.max_window) == \
        (True, True, True, 8)
    rng = np.random.default_rng(5)
    for _ in range(300):
        iou, d, med = float(np.float32(rng.uniform(0.7, 1.0))), float(np.float32(rng.uniform(0, 2))), \
            float(np.float32(rng.uniform(1, 20)))
        ref = C.is_new_keyframe(np.float32(iou), np.float32(d), np.float32(med), np.float32(0.9), np.float32(0.08))
        assert B.s3gs_keyframe_is_new(p, iou, d, med) == ref
    for _ in range(300):
        n = int(rng.integers(0, 12))
        ids = list(rng.permutation(100)[:n])
        oc = [float(np.float32(x)) for x in rng.choice([0.1, 0.29, 0.3, 0.31, 0.5, 0.5, 0.7, 0.9], n)]
        maxw = int(rng.integers(1, 10))
        q = B.s3gs_keyframe_params_default(max_window=maxw)
        ref = C.window_update(ids, [np.float32(x) for x in oc], 777, k_oc=np.float32(0.3), max_window=maxw)
        assert B.s3gs_keyframe_window_update(q, ids, oc, 777) == ref
