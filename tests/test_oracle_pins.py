"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form,
an invariant of Eq. 2/3, a library routine (scipy), a brute-force evaluation
with a different structure, or central finite differences of its own forward
(for the analytic backward of Eq. 11).
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle as O
from paper_2507_03737_gb300 import scenes

ALPHA_MIN = 1.0 / 255.0


def _single(z=5.0, s=0.05, o=0.7, col=(0.2, 0.5, 0.9), f=100.0, W=33, H=29, mu_xy=(0.0, 0.0)):
    sc = scenes.Scene(
        means=np.array([[mu_xy[0], mu_xy[1], z]], np.float32),
        log_scales=np.full((1, 3), math.log(s), np.float32),
        quats=np.array([[0.3, -0.5, 0.7, 0.2]], np.float32),  # any rotation: isotropic
        opacity_logits=np.array([math.log(o / (1 - o))], np.float32),
        colors=np.array([[col]], np.float32), sh_degree=0,
        cameras=[scenes.camera(W, H, f, f, (W - 1) / 2.0, (H - 1) / 2.0)])
    return sc


def test_single_gaussian_closed_form():
    """One isotropic Gaussian on the optical axis (Eq. 2, 3, 5 in closed form)."""
    sc = _single()
    cam = sc.cameras[0]
    z = float(sc.means[0, 2]); s = math.exp(float(sc.log_scales[0, 0]))
    o = 1.0 / (1.0 + math.exp(-float(sc.opacity_logits[0])))
    f, cx, cy = cam["fx"], cam["cx"], cam["cy"]
    var = (f * s / z) ** 2 + 0.3
    r = O.render_fwd(sc)
    W, H = cam["width"], cam["height"]
    jj, ii = np.mgrid[0:H, 0:W]
    d2 = (ii - cx) ** 2 + (jj - cy) ** 2
    q = d2 / var
    a = np.minimum(0.99, o * np.exp(-0.5 * q))
    a = np.where((q <= 9.0) & (a >= ALPHA_MIN), a, 0.0)
    a = a.reshape(-1)
    col = sc.colors[0, 0].astype(np.float64)
    np.testing.assert_allclose(r["rgb"].reshape(3, -1), col[:, None] * a[None], atol=1e-13)
    np.testing.assert_allclose(r["alpha"], a, atol=1e-13)
    np.testing.assert_allclose(r["depth"], z * a, atol=1e-12)
    X = np.stack([((ii - cx) / f).reshape(-1) * z * a, ((jj - cy) / f).reshape(-1) * z * a, z * a])
    np.testing.assert_allclose(r["pointmap"].reshape(3, -1), X, atol=1e-12)
    assert (a > 0).sum() > 20  # the footprint spans several pixels


def test_single_gaussian_closed_form_gradients():
    """dL/dcolour = sum gC alpha; dL/dlogit = sum (gC.c + gD z + gA) G o (1 - o)."""
    sc = _single(o=0.6)
    cam = sc.cameras[0]
    P = cam["width"] * cam["height"]
    rng = np.random.default_rng(3)
    gC = rng.standard_normal(3 * P); gD = rng.standard_normal(P); gA = rng.standard_normal(P)
    g = O.render_bwd(sc, d_rgb=gC, d_depth=gD, d_alpha=gA)
    fw = O.render_fwd(sc)
    a = fw["alpha"]
    z = float(sc.means[0, 2]); o = 1.0 / (1.0 + math.exp(-float(sc.opacity_logits[0])))
    col = sc.colors[0, 0].astype(np.float64)
    np.testing.assert_allclose(g["colors"][0, 0], (gC.reshape(3, -1) * a[None]).sum(1), rtol=1e-12)
    G = a / o  # no pixel is clamped (o < 0.99)
    expect = ((col[:, None] * gC.reshape(3, -1)).sum(0) + gD * z + gA) * G * o * (1 - o)
    np.testing.assert_allclose(g["opacity_logits"][0], expect.sum(), rtol=1e-10)


def test_partition_of_unity():
    """sum_k alpha_k T_k + T_final = 1 (Eq. 2 with unit colours; bg fills the rest)."""
    sc = scenes.config_scene(1, n_override=1500)
    sc.colors[:] = 1.0
    r = O.render_fwd(sc)
    for ch in range(3):
        np.testing.assert_allclose(r["rgb"].reshape(3, -1)[ch], r["alpha"], atol=1e-12)
    r2 = O.render_fwd(sc, bg=[1.0, 1.0, 1.0])
    np.testing.assert_allclose(r2["rgb"], 1.0, atol=1e-12)
    assert r["alpha"].max() > 0.9 and r["alpha"].min() >= 0.0


def test_fronto_parallel_plane():
    """Flat Gaussians at z = d: D = d * alpha and X^r = K^-1 [iD, jD, D] (Eq. 3-5)."""
    d = 4.0
    gx, gy = np.meshgrid(np.linspace(-2.6, 2.6, 53), np.linspace(-2.0, 2.0, 41))
    n = gx.size
    means = np.stack([gx.ravel(), gy.ravel(), np.full(n, d)], 1).astype(np.float32)
    ls = np.tile(np.log([0.15, 0.15, 1e-4]), (n, 1)).astype(np.float32)
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)).astype(np.float32)
    ol = np.full(n, 4.0, np.float32)
    rng = np.random.default_rng(1)
    col = rng.uniform(0, 1, (n, 1, 3)).astype(np.float32)
    cam = scenes.camera(48, 36, 40.0, 40.0, 23.5, 17.5)
    sc = scenes.Scene(means, ls, q, ol, col, 0, [cam])
    r = O.render_fwd(sc)
    np.testing.assert_allclose(r["depth"], d * r["alpha"], rtol=1e-13, atol=1e-13)
    jj, ii = np.mgrid[0:36, 0:48]
    D = r["depth"]
    pm = r["pointmap"].reshape(3, -1)
    np.testing.assert_allclose(pm[0], (ii.ravel() - 23.5) * D / 40.0, atol=1e-12)
    np.testing.assert_allclose(pm[1], (jj.ravel() - 17.5) * D / 40.0, atol=1e-12)
    np.testing.assert_allclose(pm[2], D, atol=0)
    # dense, opaque: the plane saturates and D is close to d
    assert np.median(r["alpha"]) > 0.999
    assert abs(np.median(r["depth"]) - d) < 1e-2
    assert r["alpha"].max() < 1.0 - 1e-4 + 1e-12  # the stop keeps T_final >= 1e-4


def _brute_force(proj, cam, rgb_of):
    """Unsorted O(P N^2) evaluation of Eq. 2/3: each weight is alpha_k times the
    product of (1 - alpha_l) over the Gaussians strictly in front (by (z, index)),
    blended only while that product times (1 - alpha_k) stays >= 1e-4."""
    W, H = cam["width"], cam["height"]
    valid = proj["valid"] > 0
    idx = np.nonzero(valid)[0]
    out_rgb = np.zeros((3, H * W)); out_d = np.zeros(H * W); out_a = np.zeros(H * W)
    for j in range(H):
        for i in range(W):
            dx = i - proj["u"][idx]; dy = j - proj["v"][idx]
            q = proj["A"][idx] * dx * dx + 2 * proj["B"][idx] * dx * dy + proj["C"][idx] * dy * dy
            a = np.minimum(0.99, proj["opacity"][idx] * np.exp(-0.5 * q))
            ok = (q <= 9.0) & (a >= ALPHA_MIN)
            ks = idx[ok]; ak = a[ok]; zk = proj["depth"][ks]
            acc_c = np.zeros(3); acc_d = 0.0; acc_w = 0.0
            for t in range(ks.size):
                front = (zk < zk[t]) | ((zk == zk[t]) & (ks < ks[t]))
                T = np.prod(1.0 - ak[front])
                if T * (1.0 - ak[t]) < 1e-4:
                    continue
                w = ak[t] * T
                acc_c += w * rgb_of(ks[t]); acc_d += w * zk[t]; acc_w += w
            p = j * W + i
            out_rgb[:, p] = acc_c; out_d[p] = acc_d; out_a[p] = acc_w
    return out_rgb.reshape(-1), out_d, out_a


@pytest.mark.parametrize("seed", [11, 12])
def test_brute_force_equivalence(seed):
    sc = scenes.tiny_scene(seed, n=14, width=20, height=16, max_opacity=0.99, scale=0.25)
    cam = sc.cameras[0]
    proj = O.project(sc, cam)
    rgb_of = lambda k: np.array([proj["r"][k], proj["g"][k], proj["b"][k]])
    b_rgb, b_d, b_a = _brute_force(proj, cam, rgb_of)
    r = O.render_fwd(sc)
    np.testing.assert_allclose(r["rgb"], b_rgb, atol=1e-12)
    np.testing.assert_allclose(r["depth"], b_d, atol=1e-12)
    np.testing.assert_allclose(r["alpha"], b_a, atol=1e-12)
    assert (r["n_contrib"] >= 3).any()


def test_brute_force_with_stop_rule():
    """Opaque stack: the 1e-4 stop decides what is blended (brute force agrees)."""
    n = 8
    means = np.stack([np.zeros(n), np.zeros(n), 3.0 + 0.3 * np.arange(n)], 1).astype(np.float32)
    ls = np.full((n, 3), math.log(0.3), np.float32)
    q = np.tile([1.0, 0, 0, 0], (n, 1)).astype(np.float32)
    ol = np.full(n, 4.0, np.float32)  # opacity 0.982
    rng = np.random.default_rng(5)
    col = rng.uniform(0, 1, (n, 1, 3)).astype(np.float32)
    cam = scenes.camera(12, 10, 20.0, 20.0, 5.5, 4.5)
    sc = scenes.Scene(means, ls, q, ol, col, 0, [cam])
    proj = O.project(sc, cam)
    rgb_of = lambda k: np.array([proj["r"][k], proj["g"][k], proj["b"][k]])
    b_rgb, b_d, b_a = _brute_force(proj, cam, rgb_of)
    r = O.render_fwd(sc)
    np.testing.assert_allclose(r["rgb"], b_rgb, atol=1e-12)
    np.testing.assert_allclose(r["depth"], b_d, atol=1e-12)
    assert r["n_contrib"][4 * 12 + 5] < n  # the stop cut the stack at the centre
    assert r["alpha"].max() > 0.999


def test_projection_against_pinhole_jacobian():
    """EWA 2D covariance = J_fd W Sigma W^T J_fd^T + 0.3 I with Sigma from scipy's
    rotation and J_fd the finite-difference Jacobian of the plain pinhole map."""
    sc = scenes.tiny_scene(21, n=5, n_views=2)
    for cam in sc.cameras:
        proj = O.project(sc, cam)
        T = np.asarray(cam["T_cw"], np.float64)
        Wr, t = T[:, :3], T[:, 3]
        f = np.array([cam["fx"], cam["fy"]]); c = np.array([cam["cx"], cam["cy"]])
        pin = lambda p: f * p[:2] / p[2] + c
        for g in range(sc.n):
            qw = sc.quats[g].astype(np.float64)
            R = Rotation.from_quat([qw[1], qw[2], qw[3], qw[0]]).as_matrix()
            S = np.diag(np.exp(sc.log_scales[g].astype(np.float64)))
            Sig = R @ S @ S @ R.T
            p = Wr @ sc.means[g].astype(np.float64) + t
            h = 1e-6
            Jfd = np.stack([(pin(p + h * e) - pin(p - h * e)) / (2 * h) for e in np.eye(3)], 1)
            cov = Jfd @ Wr @ Sig @ Wr.T @ Jfd.T + 0.3 * np.eye(2)
            np.testing.assert_allclose([proj["cov_a"][g], proj["cov_c"][g]], [cov[0, 0], cov[1, 1]],
                                       rtol=1e-7)
            inv = np.linalg.inv(cov)
            np.testing.assert_allclose([proj["A"][g], proj["B"][g], proj["C"][g]],
                                       [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-7)
            np.testing.assert_allclose([proj["u"][g], proj["v"][g]], pin(p), rtol=1e-12)
            assert proj["depth"][g] == pytest.approx(p[2], rel=1e-14)


def test_rotation_matches_scipy():
    rng = np.random.default_rng(2)
    for _ in range(20):
        q = rng.standard_normal(4); q /= np.linalg.norm(q)
        R = O.quat_to_rotmat(q)
        Rs = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, Rs, atol=1e-14)


def test_sh_matches_scipy_real_basis():
    """Real orthonormal SH from scipy's complex Y_l^m: Y_l,m>0 = sqrt2 (-1)^m Re Y_l^m,
    Y_l,m<0 = sqrt2 (-1)^m Im Y_l^|m|, Y_l0 = Y_l^0."""
    rng = np.random.default_rng(4)
    for _ in range(10):
        d = rng.standard_normal(3); d /= np.linalg.norm(d)
        theta = math.acos(d[2]); phi = math.atan2(d[1], d[0])
        for l in range(4):
            for m in range(-l, l + 1):
                Y = sph_harm_y(l, abs(m), theta, phi)
                if m > 0:
                    ref = math.sqrt(2) * (-1) ** m * Y.real
                elif m < 0:
                    ref = math.sqrt(2) * (-1) ** m * Y.imag
                else:
                    ref = Y.real
                assert O.sh_real(l, m, d) == pytest.approx(ref, abs=1e-12), (l, m)


def test_sh_orthonormal_by_quadrature():
    nt, nph = 24, 48
    x, w = np.polynomial.legendre.leggauss(nt)
    phis = np.arange(nph) * 2 * math.pi / nph
    basis = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    Gm = np.zeros((16, 16))
    for ct, wt in zip(x, w):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            d = np.array([st * math.cos(ph), st * math.sin(ph), ct])
            y = np.array([O.sh_real(l, m, d) for l, m in basis])
            Gm += wt * (2 * math.pi / nph) * np.outer(y, y)
    np.testing.assert_allclose(Gm, np.eye(16), atol=1e-12)


def _rigid(R0, t0, sc):
    out = sc.subset(slice(None))
    out.means = (sc.means.astype(np.float64) @ R0.T + t0).astype(np.float64)
    rq = Rotation.from_matrix(R0) * Rotation.from_quat(
        np.roll(sc.quats.astype(np.float64), -1, axis=1))
    qx = rq.as_quat()  # x, y, z, w
    out.quats = np.roll(qx, 1, axis=1) * np.linalg.norm(sc.quats.astype(np.float64), axis=1, keepdims=True)
    cams = []
    for c in sc.cameras:
        T = np.asarray(c["T_cw"], np.float64)
        Rn = T[:, :3] @ R0.T
        tn = T[:, 3] - Rn @ t0
        c2 = dict(c); c2["T_cw"] = np.concatenate([Rn, tn[:, None]], 1)
        cams.append(c2)
    out.cameras = cams
    return out


def test_rigid_motion_and_permutation_invariance():
    sc = scenes.tiny_scene(31, n=10, width=22, height=18, max_opacity=0.95)
    r0 = O.render_fwd(sc)
    R0 = Rotation.from_rotvec([0.3, -0.2, 0.5]).as_matrix(); t0 = np.array([1.0, -2.0, 0.5])
    r1 = O.render_fwd(_rigid(R0, t0, sc))
    for k in ("rgb", "depth", "pointmap", "alpha"):
        np.testing.assert_allclose(r1[k], r0[k], atol=1e-9)
    perm = np.random.default_rng(0).permutation(sc.n)
    r2 = O.render_fwd(sc.subset(perm))
    for k in ("rgb", "depth", "pointmap", "alpha"):
        np.testing.assert_allclose(r2[k], r0[k], atol=1e-13)


def test_crop_equals_window():
    """A crop (shifted principal point) equals that window of the full render."""
    sc = scenes.config_scene(1, n_override=2000)
    full = O.render_fwd(sc)
    cam = sc.cameras[0]
    x0, y0, w, h = 37, 21, 40, 30
    crop = dict(cam); crop.update(width=w, height=h, cx=cam["cx"] - x0, cy=cam["cy"] - y0)
    r = O.render_fwd(sc, cameras=[crop])
    W, H = cam["width"], cam["height"]
    for k, nch in (("rgb", 3), ("depth", 1), ("pointmap", 3), ("alpha", 1)):
        a = full[k].reshape(nch, H, W)[:, y0:y0 + h, x0:x0 + w]
        np.testing.assert_allclose(r[k].reshape(nch, h, w), a, atol=1e-9)


# ---------------- finite differences of the analytic backward (Eq. 11) ----------------

def _loss(sc, ups, cameras=None):
    r = O.render_fwd(sc, cameras=cameras)
    return sum(float(np.dot(r[k], ups[k])) for k in ("rgb", "depth", "pointmap", "alpha")), r


def _exp_left(T, tau):
    """T(tau) = Exp(tau) T with tau = (rho, phi); exact rotation for phi."""
    T = np.asarray(T, np.float64)
    Rp = Rotation.from_rotvec(tau[3:]).as_matrix()
    R = Rp @ T[:, :3]
    t = Rp @ T[:, 3] + tau[:3]
    return np.concatenate([R, t[:, None]], 1)


@pytest.mark.parametrize("seed,deg,n_views", [(41, 0, 1), (42, 3, 1), (43, 0, 2), (44, 2, 2)])
def test_backward_matches_finite_differences(seed, deg, n_views):
    sc = scenes.tiny_scene(seed, n=5, width=20, height=16, sh_degree=deg, n_views=n_views)
    # promote to float64 storage so parameter perturbations are exact
    for k in ("means", "log_scales", "quats", "opacity_logits", "colors"):
        setattr(sc, k, getattr(sc, k).astype(np.float64))
    P = sum(c["width"] * c["height"] for c in sc.cameras)
    rng = np.random.default_rng(seed)
    ups = dict(rgb=rng.standard_normal(3 * P), depth=rng.standard_normal(P),
               pointmap=rng.standard_normal(3 * P) * 0.3, alpha=rng.standard_normal(P))
    L0, r0 = _loss(sc, ups)
    assert r0["margin"].min() > 1e-4, "scene too close to a threshold; pick another seed"
    g = O.render_bwd(sc, d_rgb=ups["rgb"], d_depth=ups["depth"], d_pointmap=ups["pointmap"],
                     d_alpha=ups["alpha"])
    h = 1e-6
    for name in ("means", "log_scales", "quats", "opacity_logits", "colors"):
        arr = getattr(sc, name)
        fd = np.zeros(arr.size)
        flat = arr.reshape(-1)
        for k in range(flat.size):
            old = flat[k]
            flat[k] = old + h; Lp, _ = _loss(sc, ups)
            flat[k] = old - h; Lm, _ = _loss(sc, ups)
            flat[k] = old
            fd[k] = (Lp - Lm) / (2 * h)
        an = g[name].reshape(-1)
        err = np.linalg.norm(an - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err < 1e-6, (name, err)
        assert np.linalg.norm(fd) > 1e-3, name
    fd_tw = np.zeros((n_views, 6))
    for v in range(n_views):
        for k in range(6):
            tau = np.zeros(6)
            cams_p = [dict(c) for c in sc.cameras]; cams_m = [dict(c) for c in sc.cameras]
            tau[k] = h; cams_p[v]["T_cw"] = _exp_left(sc.cameras[v]["T_cw"], tau)
            tau[k] = -h; cams_m[v]["T_cw"] = _exp_left(sc.cameras[v]["T_cw"], tau)
            Lp, _ = _loss(sc, ups, cams_p); Lm, _ = _loss(sc, ups, cams_m)
            fd_tw[v, k] = (Lp - Lm) / (2 * h)
    err = np.linalg.norm(g["twist"] - fd_tw) / np.linalg.norm(fd_tw)
    assert err < 1e-6, err


def test_backward_background_and_alpha_terms():
    """bg and alpha gradients enter through T_final (rgb = C + T bg, alpha = 1 - T)."""
    sc = scenes.tiny_scene(51, n=4, width=16, height=12)
    for k in ("means", "log_scales", "quats", "opacity_logits", "colors"):
        setattr(sc, k, getattr(sc, k).astype(np.float64))
    P = 16 * 12
    rng = np.random.default_rng(9)
    bg = np.array([0.3, 0.6, 0.1])
    ups = dict(rgb=rng.standard_normal(3 * P), alpha=rng.standard_normal(P))
    g = O.render_bwd(sc, d_rgb=ups["rgb"], d_alpha=ups["alpha"], bg=bg)

    def L():
        r = O.render_fwd(sc, bg=bg)
        return float(np.dot(r["rgb"], ups["rgb"]) + np.dot(r["alpha"], ups["alpha"]))
    h = 1e-6
    flat = sc.opacity_logits
    fd = np.zeros(sc.n)
    for k in range(sc.n):
        old = flat[k]
        flat[k] = old + h; Lp = L(); flat[k] = old - h; Lm = L(); flat[k] = old
        fd[k] = (Lp - Lm) / (2 * h)
    np.testing.assert_allclose(g["opacity_logits"], fd, rtol=1e-6, atol=1e-9)


def test_guard_cone_culls_far_off_axis_gaussians():
    """A Gaussian just in front of the camera, far off-axis (|x/z| = 1.6 > G = 1.5), is not
    projected, even though its footprint covers the image; with the cone disabled it is."""
    sc = _single(z=0.3, s=0.6, o=0.8, mu_xy=(0.48, 0.0))  # x/z = 1.6
    try:
        O.set_guard(1.5)
        r = O.render_fwd(sc)
        assert np.abs(r["alpha"]).max() == 0.0
        O.set_guard(-1.0)
        r = O.render_fwd(sc)
        assert r["alpha"].max() > 0.1
        O.set_guard(1.7)
        assert O.render_fwd(sc)["alpha"].max() > 0.1
    finally:
        O.set_guard(1.5)
