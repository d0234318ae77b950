"""Shared helpers of the GPU parity tests (tolerances and comparisons)."""
import numpy as np

# Tolerances of the parity bar: <= 1e-4 absolute on rgb and alpha, <= 1e-4
# relative on depth and pointmap (with an absolute floor of 1e-6 where D -> 0),
# <= 1e-3 relative (L2, per tensor) on every gradient tensor.
TOL_ABS = 1e-4
TOL_REL = 1e-4
TOL_FLOOR = 1e-6
TOL_GRAD = 1e-3
MARGIN = 1e-4  # pixels whose FP64 decisions sit closer than this to a threshold are excluded


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


def compare_forward(gpu, ref, cameras, mask=None, keys=("rgb", "depth", "pointmap", "alpha"),
                    max_excluded=0.01):
    m = pixel_mask(ref) if mask is None else mask
    m3 = expand3(m, cameras)
    P = m.size
    res = {"excluded": int((~m).sum()), "pixels": P}
    if "rgb" in keys:
        res["rgb"] = float(np.abs(gpu["rgb"][m3] - ref["rgb"][m3]).max(initial=0))
        assert res["rgb"] <= TOL_ABS, res
    if "alpha" in keys:
        res["alpha"] = float(np.abs(gpu["alpha"][m] - ref["alpha"][m]).max(initial=0))
        assert res["alpha"] <= TOL_ABS, res
    if "depth" in keys:
        a, b = gpu["depth"][m], ref["depth"][m]
        bad = np.abs(a - b) > TOL_REL * np.abs(b) + TOL_FLOOR
        res["depth_bad"] = int(bad.sum())
        res["depth_rel"] = float((np.abs(a - b) / (np.abs(b) + 1e-3)).max(initial=0))
        assert res["depth_bad"] == 0, (res, _worst(a, b))
    if "pointmap" in keys:
        a, b = gpu["pointmap"][m3], ref["pointmap"][m3]
        bad = np.abs(a - b) > TOL_REL * np.abs(b) + TOL_FLOOR
        res["pointmap_bad"] = int(bad.sum())
        assert res["pointmap_bad"] == 0, (res, _worst(a, b))
    assert res["excluded"] <= max(3, max_excluded * P), res
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
