"""Pins of the pose-refinement oracle (Sec. 3.2.2, Eq. 10/11): the se(3)
exponential against the general matrix exponential, the Adam step against
PyTorch's Adam, and the refinement loop's fixed point and descent."""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from oracle import pose_oracle as PO
from paper_2507_03737_gb300 import scenes


def _hat4(tau):
    M = np.zeros((4, 4))
    M[:3, :3] = PO.hat(tau[3:])
    M[:3, 3] = tau[:3]
    return M


@pytest.mark.parametrize("theta", [0.0, 1e-7, 1e-3, 0.0099, 0.0101, 0.3, 2.0, 3.1])
def test_se3_exp_equals_matrix_exponential(theta):
    rng = np.random.default_rng(int(theta * 1e4) + 1)
    axis = rng.standard_normal(3); axis /= np.linalg.norm(axis)
    tau = np.concatenate([rng.uniform(-2, 2, 3), theta * axis])
    E = PO.se3_exp(tau)
    ref = scipy.linalg.expm(_hat4(tau))[:3, :4]
    np.testing.assert_allclose(E, ref, rtol=0, atol=1e-13)


def test_se3_exp_is_rigid_and_inverts():
    rng = np.random.default_rng(3)
    for _ in range(20):
        tau = rng.normal(0, 1, 6)
        E = PO.se3_exp(tau)
        R = E[:, :3]
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13
        I = PO.apply_left(PO.se3_exp(-tau), E)
        np.testing.assert_allclose(I, np.concatenate([np.eye(3), np.zeros((3, 1))], 1), atol=1e-13)


def test_adam_step_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    lr = np.array([1e-3] * 3 + [3e-3] * 3)
    p = torch.zeros(6, dtype=torch.float64, requires_grad=True)
    groups = [{"params": [p], "lr": 1.0}]
    opt = torch.optim.Adam(groups, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(6); v = np.zeros(6)
    for t in range(1, 6):
        g = rng.normal(0, 1, 6) * (10.0 ** rng.uniform(-3, 1, 6))
        # torch runs at lr = 1; the learning rate multiplies the whole Adam step
        delta, m, v = PO.adam_step(g, m, v, t, lr)
        with torch.no_grad():
            p.zero_()
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        np.testing.assert_allclose(delta, lr * p.detach().numpy(), rtol=1e-12, atol=0)


def _scene_and_target():
    sc = scenes.tiny_scene(5, n=12, width=32, height=24)
    tgt = O.render_fwd(sc)["rgb"]
    return sc, tgt


def test_refine_fixed_point_at_the_true_pose():
    sc, tgt = _scene_and_target()
    poses, losses, _ = PO.refine(sc, sc.cameras, tgt, iters=3)
    T0 = np.asarray(sc.cameras[0]["T_cw"], np.float64)
    for step in poses:
        np.testing.assert_array_equal(step[0], T0)
    assert losses == [0.0, 0.0, 0.0]


def test_refine_descends_from_a_perturbed_pose():
    sc, tgt = _scene_and_target()
    T0 = np.asarray(sc.cameras[0]["T_cw"], np.float64)
    start = PO.apply_left(PO.se3_exp([0.02, -0.015, 0.01, 0.01, -0.008, 0.006]), T0)
    cams = [dict(sc.cameras[0], T_cw=start)]
    poses, losses, _ = PO.refine(sc, cams, tgt, iters=30, lr_rho=2e-3, lr_phi=2e-3)
    err0 = np.linalg.norm(start - T0)
    err = np.linalg.norm(poses[-1][0] - T0)
    assert losses[-1] < 0.5 * losses[0]
    assert err < 0.5 * err0
