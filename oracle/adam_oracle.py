"""FP64 oracle of the map optimiser step of Eq. 17: the isotropic
regulariser L_iso of Eq. 16 and one Adam step over every Gaussian parameter
tensor. Test infrastructure only.

Readings taken where the paper leaves the step open:
  * s_i in Eq. 16 is the activated scale vector exp(log_scale_i); s~_i is the
    mean of its three entries; the L1 norm sums the three absolute
    deviations, and the loss sums over Gaussians as printed, weighted by
    lambda_iso (10 in the supplementary material). A caller wanting a mean
    instead scales lambda_iso by 1 / (3 |G|).
  * Its gradient treats |x| as having derivative sign(x) (0 at 0):
    dL/ds_ij = sign(s_ij - s~_i) - (1/3) sum_k sign(s_ik - s~_i), chained to
    the log-scale by ds_ij/dlog_s_ij = s_ij.
  * The optimiser is Adam (Kingma & Ba) with one step count for all tensors,
    a learning rate per tensor (the higher SH bands may take their own), and
    the gradient of L_iso added to the log-scale gradient before the step.
"""
from __future__ import annotations

import numpy as np

__all__ = ["iso_loss", "iso_grad", "adam", "map_step", "TENSORS"]

TENSORS = ("means", "log_scales", "quats", "opacity_logits", "colors")


def iso_loss(log_scales) -> float:
    s = np.exp(np.asarray(log_scales, dtype=np.float64).reshape(-1, 3))
    return float(np.abs(s - s.mean(axis=1, keepdims=True)).sum())


def iso_grad(log_scales) -> np.ndarray:
    """dL_iso/dlog_scales, shape (n, 3)."""
    s = np.exp(np.asarray(log_scales, dtype=np.float64).reshape(-1, 3))
    sg = np.sign(s - s.mean(axis=1, keepdims=True))
    ds = sg - sg.sum(axis=1, keepdims=True) / 3.0
    return ds * s


def adam(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step number t, 1-based); returns (p, m, v)."""
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    p = p - lr * (m / (1.0 - beta1 ** t)) / (np.sqrt(v / (1.0 - beta2 ** t)) + eps)
    return p, m, v


def map_step(params: dict, grads: dict, state: dict, t: int, lrs: dict, lambda_iso=10.0, beta1=0.9, beta2=0.999,
             eps=1e-8, lr_colors_rest=None):
    """One optimiser step of Eq. 17 over all Gaussian tensors. ``state`` holds
    per-tensor (m, v); lrs maps tensor name -> learning rate; colours use
    ``lr_colors_rest`` for coefficients 1.. (SH bands l >= 1) when given."""
    out_p, out_s = {}, {}
    for k in TENSORS:
        p = np.asarray(params[k], dtype=np.float64)
        g = np.asarray(grads[k], dtype=np.float64).reshape(p.shape)
        if k == "log_scales":
            g = g + lambda_iso * iso_grad(p).reshape(p.shape)
        m, v = state.get(k, (np.zeros_like(p), np.zeros_like(p)))
        lr = np.full(p.shape, float(lrs[k]))
        if k == "colors" and lr_colors_rest is not None and p.ndim == 3 and p.shape[1] > 1:
            lr[:, 1:, :] = float(lr_colors_rest)
        p, m, v = adam(p, g, m, v, t, lr, beta1, beta2, eps)
        out_p[k], out_s[k] = p, (m, v)
    return out_p, out_s
