"""Pins of the FP64 reference of the learned disentangler initialiser."""
import numpy as np

from oracle import mlp


def test_expm_of_generator_is_orthogonal():
    p = mlp.init_params(0)
    x = np.random.default_rng(0).normal(size=(8, 16))
    u, _ = mlp.forward(p, x)
    for a in u:
        assert np.abs(a.T @ a - np.eye(4)).max() < 1e-13
        assert abs(np.linalg.det(a) - 1.0) < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(3)
    for k in p:
        p[k] = p[k] + 0.1 * rng.normal(size=p[k].shape)
    x = rng.normal(size=(5, 16))
    ut = np.stack([mlp.canonical_target(np.linalg.qr(rng.normal(size=(4, 4)))[0]) for _ in range(5)])
    loss, g = mlp.loss_and_grad(p, x, ut)
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + 1e-6
            lp, _ = mlp.loss_and_grad(p, x, ut)
            flat[idx] = old - 1e-6
            lm, _ = mlp.loss_and_grad(p, x, ut)
            flat[idx] = old
            fd = (lp - lm) / 2e-6
            assert abs(fd - g[k].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), k


def test_adam_reduces_loss():
    rng = np.random.default_rng(2)
    p = mlp.init_params(1)
    x = rng.normal(size=(16, 16))
    ut = np.stack([mlp.canonical_target(np.linalg.qr(rng.normal(size=(4, 4)))[0]) for _ in range(16)])
    opt = mlp.Adam(p, lr=3e-3)
    l0, _ = mlp.loss_and_grad(p, x, ut)
    for _ in range(60):
        l, g = mlp.loss_and_grad(p, x, ut)
        opt.step(p, g)
    assert l < 0.5 * l0
