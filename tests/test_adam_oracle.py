"""Pins of the map-optimiser oracle (Eq. 16 and the Adam step of Eq. 17):
the L_iso gradient against finite differences and PyTorch autograd, its
closed-form special cases, and the Adam step against torch.optim.Adam."""
import numpy as np
import pytest

from oracle import adam_oracle as A


def test_iso_zero_for_isotropic_scales():
    ls = np.log(np.array([[0.1, 0.1, 0.1], [2.0, 2.0, 2.0]]))
    assert A.iso_loss(ls) == 0.0
    np.testing.assert_array_equal(A.iso_grad(ls), np.zeros((2, 3)))


def test_iso_closed_form_two_equal_one_larger():
    # s = (1, 1, 4): mean 2, loss = 1 + 1 + 2 = 4; signs (-,-,+) sum -1:
    # dL/ds = (-1 + 1/3, -1 + 1/3, 1 + 1/3), times s
    ls = np.log(np.array([[1.0, 1.0, 4.0]]))
    assert abs(A.iso_loss(ls) - 4.0) < 1e-12
    np.testing.assert_allclose(A.iso_grad(ls), [[-2 / 3, -2 / 3, 16 / 3]], rtol=1e-12)


def test_iso_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    ls = rng.normal(np.log(0.05), 0.5, (50, 3))
    g = A.iso_grad(ls)
    h = 1e-6
    for i in range(50):
        for j in range(3):
            e = np.zeros_like(ls); e[i, j] = h
            fd = (A.iso_loss(ls + e) - A.iso_loss(ls - e)) / (2 * h)
            assert abs(fd - g[i, j]) <= 1e-6 * max(1.0, abs(g[i, j]))


def test_iso_gradient_matches_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    ls = rng.normal(0.0, 1.0, (200, 3))
    t = torch.tensor(ls, dtype=torch.float64, requires_grad=True)
    s = torch.exp(t)
    (s - s.mean(dim=1, keepdim=True)).abs().sum().backward()
    np.testing.assert_allclose(A.iso_grad(ls), t.grad.numpy(), rtol=1e-12, atol=1e-15)


def test_map_step_matches_torch_adam_per_group():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    n, nc = 40, 4
    params = dict(means=rng.normal(0, 1, (n, 3)), log_scales=rng.normal(-3, 0.5, (n, 3)),
                  quats=rng.normal(0, 1, (n, 4)), opacity_logits=rng.normal(0, 1, n),
                  colors=rng.normal(0, 0.3, (n, nc, 3)))
    lrs = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, opacity_logits=5e-2, colors=2.5e-3)
    lam = 10.0
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in params.items()}
    groups = [{"params": [tp[k]], "lr": lrs[k]} for k in ("means", "log_scales", "quats", "opacity_logits")]
    dc = torch.tensor(params["colors"][:, :1], dtype=torch.float64, requires_grad=True)
    rest = torch.tensor(params["colors"][:, 1:], dtype=torch.float64, requires_grad=True)
    groups += [{"params": [dc], "lr": lrs["colors"]}, {"params": [rest], "lr": lrs["colors"] / 20}]
    opt = torch.optim.Adam(groups, betas=(0.9, 0.999), eps=1e-8)
    p_or, st = params, {}
    for t in range(1, 5):
        grads = {k: rng.normal(0, 1, v.shape) * 10.0 ** rng.uniform(-3, 0) for k, v in params.items()}
        p_or, st = A.map_step(p_or, grads, st, t, lrs, lambda_iso=lam, lr_colors_rest=lrs["colors"] / 20)
        for k in ("means", "log_scales", "quats", "opacity_logits"):
            tp[k].grad = torch.tensor(grads[k], dtype=torch.float64)
        tp["log_scales"].grad += lam * torch.tensor(A.iso_grad(tp["log_scales"].detach().numpy()))
        dc.grad = torch.tensor(grads["colors"][:, :1]); rest.grad = torch.tensor(grads["colors"][:, 1:])
        opt.step()
        for k in ("means", "log_scales", "quats", "opacity_logits"):
            np.testing.assert_allclose(p_or[k], tp[k].detach().numpy(), rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(p_or["colors"][:, :1], dc.detach().numpy(), rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(p_or["colors"][:, 1:], rest.detach().numpy(), rtol=1e-13, atol=1e-15)
