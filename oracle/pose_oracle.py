"""FP64 oracle of photometric pose refinement (Sec. 3.2.2, Eq. 10 and 11): the
se(3) exponential, the optimiser step on the twist and the refinement loop
built on the renderer oracle. Test infrastructure only.

Readings taken where the paper leaves the loop open:
  * The pose is world-to-camera T_cw, perturbed on the left, T(tau) =
    Exp(tau) T_cw with tau = (rho, phi) (rho: translation part, phi: rotation
    vector), as in the renderer's twist gradient.
  * Each iteration renders the view at its current pose, takes the L1
    photometric loss of Eq. 10 as the mean over pixels and colour channels of
    w(x) |I(x) - Ibar(x)| (w = the caller's per-pixel weight, the paper's
    emphasis on edges and valid regions), differentiates it with respect to
    tau at tau = 0, and takes one Adam step on tau starting from tau = 0; the
    pose is then retracted, T_cw <- Exp(delta) T_cw, so the twist is always
    linearised at the current pose (Eq. 11). The Adam moments persist across
    iterations; the learning rates of rho and phi are inputs.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O

__all__ = ["hat", "se3_exp", "adam_step", "apply_left", "refine"]


def hat(phi) -> np.ndarray:
    """Skew-symmetric matrix [phi]_x (so that [phi]_x p = phi x p)."""
    x, y, z = (float(v) for v in phi)
    return np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])


def se3_exp(tau) -> np.ndarray:
    """Exp of tau = (rho, phi) as the 3x4 [R | V rho], from the closed forms
    R = I + a K + b K^2 and V = I + b K + c K^2 with K = [phi]_x, theta = |phi|,
    a = sin(theta)/theta, b = (1 - cos(theta))/theta^2, c = (theta - sin(theta))/theta^3
    (their Taylor series for small theta)."""
    tau = np.asarray(tau, dtype=np.float64).reshape(6)
    rho, phi = tau[:3], tau[3:]
    th2 = float(phi @ phi)
    th = math.sqrt(th2)
    K = hat(phi)
    if th < 1e-2:
        a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0 - th2 ** 3 / 5040.0
        b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0 - th2 ** 3 / 40320.0
        c = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0 - th2 ** 3 / 362880.0
    else:
        a = math.sin(th) / th
        b = (1.0 - math.cos(th)) / th2
        c = (th - math.sin(th)) / (th2 * th)
    K2 = K @ K
    R = np.eye(3) + a * K + b * K2
    V = np.eye(3) + b * K + c * K2
    return np.concatenate([R, (V @ rho)[:, None]], axis=1)


def apply_left(E, T) -> np.ndarray:
    """E T for 3x4 rigid transforms."""
    E = np.asarray(E, dtype=np.float64).reshape(3, 4)
    T = np.asarray(T, dtype=np.float64).reshape(3, 4)
    return np.concatenate([E[:, :3] @ T[:, :3], (E[:, :3] @ T[:, 3] + E[:, 3])[:, None]], axis=1)


def adam_step(g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step from a parameter at 0 (Kingma & Ba, Algorithm 1): returns
    (delta, m, v) for step number t (1-based), elementwise learning rates lr."""
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    delta = -np.asarray(lr, dtype=np.float64) * m_hat / (np.sqrt(v_hat) + eps)
    return delta, m, v


def refine(scene, cameras, target_rgb, iters, lr_rho=1e-3, lr_phi=1e-3, weight=None, beta1=0.9, beta2=0.999,
           eps=1e-8, near_z=0.2):
    """Pose refinement of every view (independently) for ``iters`` iterations.
    target_rgb: packed planar rgb of all views; weight: packed per-pixel weights
    (None = 1). Returns the list of 3x4 poses after each iteration (per view),
    the loss before each iteration and the twist gradients of each iteration."""
    cams = [dict(c, T_cw=np.asarray(c["T_cw"], dtype=np.float64).reshape(3, 4)) for c in cameras]
    V = len(cams)
    P = sum(c["width"] * c["height"] for c in cams)
    t_rgb = np.asarray(target_rgb, dtype=np.float64)
    w = np.ones(P) if weight is None else np.asarray(weight, dtype=np.float64)
    lr = np.array([lr_rho] * 3 + [lr_phi] * 3)
    m = np.zeros((V, 6)); v = np.zeros((V, 6))
    poses, losses, grads = [], [], []
    for it in range(1, iters + 1):
        out = O.render_fwd(scene, cameras=cams, near_z=near_z)
        r = out["rgb"] - t_rgb
        # per-pixel weight broadcast over the three planes of each view
        w3 = np.concatenate([np.tile(w[o:o + c["width"] * c["height"]], 3)
                             for o, c in zip(O.pixel_offsets(cams)[:-1], cams)])
        losses.append(float((w3 * np.abs(r)).sum() / (3.0 * P)))
        d_rgb = w3 * np.sign(r) / (3.0 * P)
        g = O.render_bwd(scene, d_rgb=d_rgb, cameras=cams, near_z=near_z)["twist"]
        grads.append(g.copy())
        step = []
        for k in range(V):
            delta, m[k], v[k] = adam_step(g[k], m[k], v[k], it, lr, beta1, beta2, eps)
            cams[k] = dict(cams[k], T_cw=apply_left(se3_exp(delta), cams[k]["T_cw"]))
            step.append(cams[k]["T_cw"].copy())
        poses.append(step)
    return poses, losses, grads
