"""Shared helpers of the GPU parity tests (tolerances and comparisons)."""
import json
import os

import numpy as np

# Tolerances of the parity bar: <= 1e-4 absolute on rgb and alpha, <= 1e-4
# relative on depth and pointmap (with an absolute floor of 1e-6 where D -> 0),
# <= 1e-3 relative (L2, per tensor) on every gradient tensor.
TOL_ABS = 1e-4
TOL_REL = 1e-4
TOL_FLOOR = 1e-6
TOL_GRAD = 1e-3
MARGIN = 1e-5  # pixels whose FP64 decisions sit closer than this (relative) to a threshold are excluded


def report(name, res):
    """Record a parity comparison's exclusion counts: printed (pytest -s shows it) and,
    when S3GS_PARITY_LOG names a file, appended to it as one JSON line."""
    line = {"test": name, **{k: v for k, v in res.items() if isinstance(v, (int, float, str))}}
    print("PARITY " + json.dumps(line))
    path = os.environ.get("S3GS_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(line) + "\n")
    return res


def expand3(x, cameras):
    """Per-pixel array (P,) -> packed 3-channel layout (3P,): view v, channel c, pixel p."""
    out, off = [], 0
    for c in cameras:
        hw = c["width"] * c["height"]
        out.append(np.tile(x[off:off + hw], 3))
        off += hw
    return np.concatenate(out)


def planes(x, cameras, ch):
    """Split a packed output into per-view arrays of shape (ch, H, W)."""
    out, off = [], 0
    for c in cameras:
        hw = c["width"] * c["height"]
        out.append(x[ch * off: ch * (off + hw)].reshape(ch, c["height"], c["width"]))
        off += hw
    return out


def pixel_mask(ref, thresh=MARGIN):
    return ref["margin"] > thresh


def _pixel_fails(gpu, ref, cameras, sel):
    """Per pixel: does any output of the pixel exceed the parity tolerance? (sel: bool [P])"""
    bad = np.zeros(sel.size, bool)
    off = 0
    for c in cameras:
        hw = c["width"] * c["height"]
        s1 = slice(off, off + hw)
        for k, ch in (("rgb", 3), ("pointmap", 3), ("depth", 1), ("alpha", 1)):
            if k not in gpu or k not in ref:
                continue
            a = gpu[k][ch * off: ch * (off + hw)].reshape(ch, hw).astype(np.float64)
            b = ref[k][ch * off: ch * (off + hw)].reshape(ch, hw)
            if k in ("rgb", "alpha"):
                e = np.abs(a - b) > TOL_ABS
            else:
                e = np.abs(a - b) > TOL_REL * np.abs(b) + TOL_FLOOR
            bad[s1] |= e.any(axis=0)
        off += hw
    return bad & sel


def compare_forward(gpu, ref, cameras, mask=None, keys=("rgb", "depth", "pointmap", "alpha"),
                    max_excluded=0.002, name=None):
    """Forward outputs against the oracle on the pixels whose decisions lie outside the
    margin band; at most max(3, max_excluded * pixels) pixels may be excluded. The
    result also counts, for the record, the pixels a band ten times narrower would add
    and how many of those would break the tolerance; it is reported (see report)
    under ``name``, by default the running test's id."""
    m = pixel_mask(ref) if mask is None else mask
    m3 = expand3(m, cameras)
    P = m.size
    res = {"excluded": int((~m).sum()), "pixels": P, "max_excluded": int(max(3, max_excluded * P))}
    if mask is None and "margin" in ref:
        narrow = (ref["margin"] > MARGIN / 10) & ~m
        res["narrow_band_added"] = int(narrow.sum())
        res["narrow_band_fail"] = int(_pixel_fails(gpu, ref, cameras, narrow).sum())
    worst = {}
    if "rgb" in keys:
        res["rgb"] = float(np.abs(gpu["rgb"][m3] - ref["rgb"][m3]).max(initial=0))
    if "alpha" in keys:
        res["alpha"] = float(np.abs(gpu["alpha"][m] - ref["alpha"][m]).max(initial=0))
    if "depth" in keys:
        a, b = gpu["depth"][m], ref["depth"][m]
        bad = np.abs(a - b) > TOL_REL * np.abs(b) + TOL_FLOOR
        res["depth_bad"] = int(bad.sum())
        res["depth_rel"] = float((np.abs(a - b) / (np.abs(b) + 1e-3)).max(initial=0))
        if bad.any():
            worst["depth"] = _worst(a, b)
    if "pointmap" in keys:
        a, b = gpu["pointmap"][m3], ref["pointmap"][m3]
        bad = np.abs(a - b) > TOL_REL * np.abs(b) + TOL_FLOOR
        res["pointmap_bad"] = int(bad.sum())
        if bad.any():
            worst["pointmap"] = _worst(a, b)
    if name is None:
        name = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    report(name, res)
    assert res.get("rgb", 0.0) <= TOL_ABS, res
    assert res.get("alpha", 0.0) <= TOL_ABS, res
    assert res.get("depth_bad", 0) == 0, (res, worst)
    assert res.get("pointmap_bad", 0) == 0, (res, worst)
    assert res["excluded"] <= res["max_excluded"], res
    return res


def _worst(a, b):
    i = int(np.argmax(np.abs(a - b)))
    return dict(i=i, gpu=float(a[i]), ref=float(b[i]))


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1); b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def compare_grads(gpu, ref, keys=("means", "log_scales", "quats", "opacity_logits", "colors", "twist"),
                  tol=TOL_GRAD):
    errs = {k: rel_l2(gpu[k], ref[k]) for k in keys if k in gpu}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, errs
    return errs


def upstream(cameras, seed, mask=None):
    """Seeded N(0,1) upstream gradients, zeroed on excluded pixels (all of a pixel's
    backward terms are linear in its upstream gradients, so this removes the pixel)."""
    P = sum(c["width"] * c["height"] for c in cameras)
    rng = np.random.default_rng(seed)
    ups = dict(d_rgb=rng.standard_normal(3 * P), d_depth=rng.standard_normal(P),
               d_pointmap=rng.standard_normal(3 * P), d_alpha=rng.standard_normal(P))
    if mask is not None:
        m = mask.astype(np.float64)
        m3 = expand3(m, cameras)
        ups["d_rgb"] = ups["d_rgb"] * m3
        ups["d_pointmap"] = ups["d_pointmap"] * m3
        ups["d_depth"] = ups["d_depth"] * m
        ups["d_alpha"] = ups["d_alpha"] * m
    return ups
