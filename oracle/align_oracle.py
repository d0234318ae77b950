"""FP64 oracle of the pointmap scale alignment (Sec. 3.3.1 and Algorithm 1 of the
supplementary material), the pointmap replacement (Eq. 14) and the remedial
scale factor (supplementary, Sec. "Patch-based Scale Alignment").

Test infrastructure only: the product library never imports this module. It is
written from the paper's description, step by step, in plain numpy with
explicit per-patch loops, in float64.

Pointmaps are (3, H, W) arrays (x, y, z planes of one view), the layout in
which the renderer emits its pointmap (Eq. 5).

Readings taken where the paper leaves the computation open:
  * A patch is a P x P block of the H x W grid, starting at pixel (0, 0);
    where H or W is not a multiple of P the last row/column of patches is
    smaller and is used as it is.
  * The mean mu and standard deviation sigma of a patch are taken jointly over
    every coordinate value of every point in it (3 * rows * cols values); the
    standard deviation is the population one (divisor = number of values).
  * A patch is a candidate when |mu_r - mu_p| < delta_mu * mu_p and
    |sigma_r - sigma_p| < delta_sigma * sigma_p (strict, as printed).
  * A point x of a candidate patch is a correct point when the Euclidean norm
    of the difference of its normalised 3-vectors is below eps_r.
  * The correct-point set CP is rebuilt at every iteration (a set of pixels;
    each pixel once), and the scale is the ratio of the mean coordinate value
    of X^r over CP to that of the ORIGINAL X^p over CP (so that sigma' * X^p,
    not sigma' * X^p_iter, is the aligned map, as the algorithm's update
    X^p_{iter+1} = sigma' * X^p states). Because the algorithm recomputes the
    ratio after each candidate patch from the growing CP, its value after the
    patch loop is the ratio over the whole CP of the iteration; if CP is empty
    the previous sigma' stays.
  * Iterations start from sigma' = sigma_init (1 in Algorithm 1; the remedial
    factor when the remedy re-runs one iteration).
  * |CP| is insufficient when |CP| < tau * N_p with N_p = H * W.
  * Eq. 14 compares Euclidean norms per point: X^r(x) is kept when
    ||X^r(x) - Xhat^p(x)|| <= eps_m * ||Xhat^p(x)||, else replaced by Xhat^p(x).
  * The remedial factor is the ratio of the mean coordinate value of the
    aligned adjacent-keyframe pointmap over the matched points to that of the
    current pointmap over its matched points; the matches themselves (a
    learned feature matcher) are an input.
"""
from __future__ import annotations

import numpy as np

__all__ = ["patch_grid", "patch_stats", "align", "replace", "remedy_scale", "DEFAULTS"]

# Hyperparameters of the supplementary material's parameter table, and eps_m.
DEFAULTS = dict(P=10, delta_mu=0.3, delta_sigma=0.3, eps_r=0.1, max_iter=3, tau=0.01, eps_m=0.15)


def patch_grid(H: int, W: int, P: int):
    """Row and column slices of the P x P patches (edge patches may be smaller)."""
    rows = [slice(y, min(y + P, H)) for y in range(0, H, P)]
    cols = [slice(x, min(x + P, W)) for x in range(0, W, P)]
    return rows, cols


def patch_stats(X: np.ndarray, rs: slice, cs: slice):
    """Joint mean and population standard deviation of all coordinate values of a patch."""
    vals = np.asarray(X[:, rs, cs], dtype=np.float64).reshape(-1)
    mu = vals.sum() / vals.size
    sd = np.sqrt(((vals - mu) ** 2).sum() / vals.size)
    return mu, sd


def align(Xr, Xp, P=10, delta_mu=0.3, delta_sigma=0.3, eps_r=0.1, max_iter=3, tau=0.01, sigma_init=1.0):
    """Algorithm 1 on one view. Returns a dict with the final scale ``sigma``, the
    per-iteration scales, |CP| and the CP mask of the last iteration, the
    insufficiency flag, decision margins (relative distances of every
    candidate test and every correct-point test from its threshold) for the
    last iteration, and the smallest of each kind for every iteration."""
    Xr = np.asarray(Xr, dtype=np.float64)
    Xp = np.asarray(Xp, dtype=np.float64)
    _, H, W = Xr.shape
    rows, cols = patch_grid(H, W, P)
    sigma = float(sigma_init)
    history = []
    min_margins = []   # per iteration: smallest patch margin, smallest point margin
    cp = np.zeros((H, W), dtype=bool)
    patch_margin = np.full((len(rows), len(cols)), np.inf)
    point_margin = np.full((H, W), np.inf)
    for _ in range(max_iter):
        Xp_it = sigma * Xp
        cp = np.zeros((H, W), dtype=bool)
        patch_margin = np.full((len(rows), len(cols)), np.inf)
        point_margin = np.full((H, W), np.inf)
        for i, rs in enumerate(rows):
            for j, cs in enumerate(cols):
                mu_r, sd_r = patch_stats(Xr, rs, cs)
                mu_p, sd_p = patch_stats(Xp_it, rs, cs)
                lim_mu, lim_sd = delta_mu * mu_p, delta_sigma * sd_p
                # signed relative distances from the two thresholds (> 0: test passes)
                m_mu = (lim_mu - abs(mu_r - mu_p)) / max(abs(lim_mu), 1e-300)
                m_sd = (lim_sd - abs(sd_r - sd_p)) / max(abs(lim_sd), 1e-300)
                candidate = abs(mu_r - mu_p) < lim_mu and abs(sd_r - sd_p) < lim_sd
                if candidate:
                    patch_margin[i, j] = min(m_mu, m_sd)
                else:  # the decision is as safe as the clearest failing test
                    patch_margin[i, j] = max(-m for m in (m_mu, m_sd) if m <= 0)
                if not candidate:
                    continue
                # normalise both patches and test every point of the patch
                nr = (Xr[:, rs, cs] - mu_r) / sd_r
                np_ = (Xp_it[:, rs, cs] - mu_p) / sd_p
                d = np.sqrt(((nr - np_) ** 2).sum(axis=0))
                cp[rs, cs] = d < eps_r
                point_margin[rs, cs] = np.abs(eps_r - d) / eps_r
        min_margins.append((float(patch_margin.min()), float(point_margin.min())))
        if cp.any():
            num = Xr[:, cp].sum()
            den = Xp[:, cp].sum()
            sigma = float(num / den)
        history.append(sigma)
    n_cp = int(cp.sum())
    return dict(sigma=sigma, history=history, n_cp=n_cp, cp=cp,
                insufficient=bool(n_cp < tau * H * W), patch_margin=patch_margin,
                point_margin=point_margin, min_margins=min_margins)


def replace(Xr, Xp, sigma: float, eps_m=0.15):
    """Eq. 14 with Xhat^p = sigma * X^p. Returns (Xhat^r, Xhat^p, replaced mask, margin)."""
    Xr = np.asarray(Xr, dtype=np.float64)
    Xp_hat = float(sigma) * np.asarray(Xp, dtype=np.float64)
    err = np.sqrt(((Xr - Xp_hat) ** 2).sum(axis=0))
    lim = eps_m * np.sqrt((Xp_hat ** 2).sum(axis=0))
    replaced = err > lim
    out = np.where(replaced[None], Xp_hat, Xr)
    margin = np.abs(lim - err) / np.maximum(lim, 1e-300)
    return out, Xp_hat, replaced, margin


def remedy_scale(X_ak_hat, X_n, matches) -> float:
    """Remedial factor from matched pixels: matches is an (M, 2) array of flat
    pixel indices (index in the adjacent keyframe's map, index in the current map)."""
    A = np.asarray(X_ak_hat, dtype=np.float64).reshape(3, -1)
    B = np.asarray(X_n, dtype=np.float64).reshape(3, -1)
    m = np.asarray(matches, dtype=np.int64).reshape(-1, 2)
    return float(A[:, m[:, 0]].sum() / B[:, m[:, 1]].sum())
