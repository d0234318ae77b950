"""Pins of the scale-alignment / replacement oracle (Algorithm 1, Eq. 14).

Each expected value here follows from a construction whose answer is known
without running the algorithm: exact rescalings, planted outlier patches and
points, closed-form statistics, and invariances of the method.
"""
import numpy as np
import pytest

from oracle import align_oracle as A


def _positive_map(rng, H, W):
    """A plausible camera-frame pointmap: z in [5, 50], x and y spread around it."""
    z = rng.uniform(5.0, 50.0, (H, W))
    x = rng.uniform(-0.6, 0.6, (H, W)) * z
    y = rng.uniform(-0.2, 0.3, (H, W)) * z
    return np.stack([x, y, z])


def test_population_std_reading():
    # values {1, 3} repeated: mean 2, population std 1 (the sample std would be sqrt(6/5))
    X = np.array([[[1.0, 3.0]], [[1.0, 3.0]], [[1.0, 3.0]]])
    mu, sd = A.patch_stats(X, slice(0, 1), slice(0, 2))
    assert mu == 2.0 and sd == 1.0


def test_patch_grid_keeps_ragged_edges():
    rows, cols = A.patch_grid(13, 21, 10)
    assert [(s.start, s.stop) for s in rows] == [(0, 10), (10, 13)]
    assert [(s.start, s.stop) for s in cols] == [(0, 10), (10, 20), (20, 21)]


@pytest.mark.parametrize("s", [0.8, 1.0, 1.2])
def test_exact_rescaling_recovers_the_scale(s):
    rng = np.random.default_rng(1)
    Xr = _positive_map(rng, 23, 37)      # ragged in both directions
    Xp = Xr / s
    out = A.align(Xr, Xp)
    assert abs(out["sigma"] - s) <= 1e-12 * s
    assert out["n_cp"] == 23 * 37 and not out["insufficient"]
    assert all(abs(h - s) <= 1e-12 * s for h in out["history"])


def test_scale_outside_the_gate_finds_no_candidates_and_remedy_recovers_it():
    rng = np.random.default_rng(2)
    Xr = _positive_map(rng, 20, 30)
    Xp = Xr / 1.5                        # |mu_r - mu_p| = 0.5 mu_p: no patch passes
    out = A.align(Xr, Xp)
    assert out["sigma"] == 1.0 and out["n_cp"] == 0 and out["insufficient"]
    # one more iteration from a remedial factor within the gate recovers 1.5
    again = A.align(Xr, Xp, sigma_init=1.4, max_iter=1)
    assert abs(again["sigma"] - 1.5) <= 1e-12
    assert again["n_cp"] == 600


def test_planted_outliers_define_the_correct_points():
    """Good patches hold X^p = X^r / s except a few planted deviating points;
    bad patches hold unrelated values. CP = good patches minus deviators, so the
    scale is s exactly at every iteration (a ratio against the rescaled X^p_iter
    instead of the original X^p would return 1 at iteration 2)."""
    rng = np.random.default_rng(3)
    P, s = 10, 1.1
    H, W = 30, 40
    Xr = _positive_map(rng, H, W)
    Xp = Xr / s
    bad = [(0, 1), (2, 3)]
    for (i, j) in bad:
        Xp[:, i * P:(i + 1) * P, j * P:(j + 1) * P] = _positive_map(rng, P, P) * 4.0
    deviators = [(5, 5), (12, 27), (25, 8)]
    for (y, x) in deviators:
        Xp[2, y, x] += 12.0              # far off in depth
    expect = np.ones((H, W), dtype=bool)
    for (i, j) in bad:
        expect[i * P:(i + 1) * P, j * P:(j + 1) * P] = False
    for (y, x) in deviators:
        expect[y, x] = False
    out = A.align(Xr, Xp, P=P)
    np.testing.assert_array_equal(out["cp"], expect)
    assert abs(out["sigma"] - s) <= 1e-12 * s
    assert len(out["history"]) == 3 and all(abs(h - s) <= 1e-12 * s for h in out["history"])


def test_insufficient_threshold_is_tau_times_pixels():
    rng = np.random.default_rng(4)
    Xr = _positive_map(rng, 20, 20)
    Xp = Xr.copy()
    Xp[:, 10:, :] = _positive_map(rng, 10, 20) * 5.0   # half the patches are bad
    Xp[:, :10, 10:] = _positive_map(rng, 10, 10) * 5.0  # three quarters bad
    out = A.align(Xr, Xp)
    assert out["n_cp"] == 100
    assert not A.align(Xr, Xp, tau=0.25)["insufficient"]       # 100 >= 0.25 * 400
    assert A.align(Xr, Xp, tau=0.2501)["insufficient"]


def test_invariances_uniform_scaling_and_patch_permutation():
    rng = np.random.default_rng(5)
    Xr = _positive_map(rng, 30, 30)
    Xp = Xr / 1.15 * (1.0 + rng.normal(0.0, 0.03, Xr.shape))   # noisy: CP is a strict subset
    base = A.align(Xr, Xp)
    assert 0 < base["n_cp"] < 900
    scaled = A.align(Xr * 3.0, Xp * 3.0)
    np.testing.assert_array_equal(scaled["cp"], base["cp"])
    assert abs(scaled["sigma"] - base["sigma"]) <= 1e-12
    # swap patch blocks (0,0) <-> (2,1) in both maps
    def swap(X):
        Y = X.copy()
        a, b = (slice(0, 10), slice(0, 10)), (slice(20, 30), slice(10, 20))
        Y[:, a[0], a[1]], Y[:, b[0], b[1]] = X[:, b[0], b[1]], X[:, a[0], a[1]]
        return Y
    perm = A.align(swap(Xr), swap(Xp))
    assert perm["n_cp"] == base["n_cp"]
    np.testing.assert_array_equal(swap(base["cp"][None])[0], perm["cp"])
    assert abs(perm["sigma"] - base["sigma"]) <= 1e-12 * base["sigma"]


def test_replacement_thresholds_and_idempotence():
    rng = np.random.default_rng(6)
    Xp = _positive_map(rng, 8, 9)
    s = 1.25
    Xr = s * Xp * 1.10                   # 10 % off: kept (<= 15 %)
    Xr[:, 0, :] = s * Xp[:, 0, :] * 1.20  # 20 % off: replaced
    out, Xp_hat, replaced, margin = A.replace(Xr, Xp, s)
    assert replaced[0].all() and not replaced[1:].any()
    np.testing.assert_allclose(Xp_hat, s * Xp, rtol=0, atol=0)
    np.testing.assert_array_equal(out[:, 0], Xp_hat[:, 0])
    np.testing.assert_array_equal(out[:, 1:], Xr[:, 1:])
    again, _, rep2, _ = A.replace(out, Xp, s)
    np.testing.assert_array_equal(again, out)
    assert not rep2.any()
    assert np.all(margin > 0.3)


def test_replacement_is_per_point_not_per_coordinate():
    # x off by 100 % of itself but the point as a whole within 15 %: kept
    Xp = np.array([[[0.1]], [[0.0]], [[10.0]]])
    Xr = np.array([[[0.2]], [[0.0]], [[10.0]]])
    _, _, replaced, _ = A.replace(Xr, Xp, 1.0)
    assert not replaced.any()


def test_remedy_scale_from_matches():
    rng = np.random.default_rng(7)
    X_ak = _positive_map(rng, 12, 16)
    perm = rng.permutation(12 * 16)
    X_n = (X_ak.reshape(3, -1)[:, perm] / 0.7).reshape(3, 12, 16)
    # pixel perm[k] of the keyframe map is pixel k of the current map
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    idx = rng.choice(perm.size, 50, replace=False)
    matches = np.stack([idx, inv[idx]], axis=1)
    assert abs(A.remedy_scale(X_ak, X_n, matches) - 0.7) <= 1e-12
