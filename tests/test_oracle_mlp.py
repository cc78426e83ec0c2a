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


def test_adam_two_steps_match_hand_derived_values():
    """Two Adam steps (Kingma and Ba 2015: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    p -= lr m/(1 - b1^t) / (sqrt(v/(1 - b2^t)) + eps), b1 = 0.9, b2 = 0.999, eps = 1e-8,
    lr = 0.01) on a three-parameter toy, worked out by hand to 40 digits:
      step 1, g = (0.1, -0.2, 0.3): m = (0.01, -0.02, 0.03), v = (1e-5, 4e-5, 9e-5), the
        bias-corrected step is lr g / (|g| + eps) for every entry;
      step 2, g = (-0.05, 0.4, 0): m = (0.004, 0.022, 0.027),
        v = (1.249e-5, 1.9996e-4, 8.991e-5), corrections 1 - 0.9^2 = 0.19 and
        1 - 0.999^2 = 0.001999.
    A dropped bias correction moves step 1 by about 3.16 lr instead of lr; swapped
    b1/b2 or eps under the square root change the step-2 (or step-1) values."""
    p = {"w": np.array([1.0, -2.0, 0.5])}
    opt = mlp.Adam(p, lr=0.01)
    opt.step(p, {"w": np.array([0.1, -0.2, 0.3])})
    step1 = np.array([0.9900000009999999000000099999990000001000, -1.990000000499999975000001249999937500003,
                      0.4900000003333333222222225925925802469140])
    assert np.abs(p["w"] - step1).max() < 1e-15
    opt.step(p, {"w": np.array([-0.05, 0.4, 0.0])})
    step2 = np.array([0.9873366309403390703755550369949895370613, -1.993661035654603704419413438190278103869,
                      0.4832994181079153989809021434622533999186])
    assert np.abs(p["w"] - step2).max() < 1e-15
