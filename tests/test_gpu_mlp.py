"""Learned disentangler start: GPU FP32 kernels against the FP64 oracle
(forward, loss, gradients through expm), training, and the gain over the
plain identity start judged by the method's own energy E_k."""
import numpy as np
import pytest

from inputs import raw_tree_tensors
from oracle import mlp as omlp
from oracle.tree import Tree
from tests.gpu_util import lib_and_ctx

pytestmark = pytest.mark.gpu


def _flat(p):
    return np.concatenate([p[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


def _unflat(v):
    out, o = {}, 0
    for k, shp in (("W1", (128, 16)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (16, 128)),
                   ("b3", (16,))):
        n = int(np.prod(shp))
        out[k] = v[o:o + n].reshape(shp).astype(np.float64)
        o += n
    return out


def _batch(rng, B):
    x = rng.normal(size=(B, 16))
    ut = np.stack([omlp.canonical_target(np.linalg.qr(rng.normal(size=(4, 4)))[0]) for _ in range(B)])
    return x, ut


@pytest.mark.parametrize("B", [24, 300])  # 300: more samples than one block of the head kernel
def test_forward_loss_and_gradients_match_oracle(B):
    attn, ctx = lib_and_ctx()
    assert attn.attn_mlp_param_count() == 16 * 128 + 128 + 128 * 128 + 128 + 128 * 16 + 16
    rng = np.random.default_rng(0)
    p = omlp.init_params(3)
    for k in p:
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    pf = _flat(p)
    p32 = _unflat(pf)  # the oracle sees the same (FP32-rounded) parameters
    x, ut = _batch(rng, B)
    m = attn.attn_mlp_create(ctx, pf)
    u = attn.attn_mlp_predict(m, x)
    u_ref, _ = omlp.forward(p32, x)
    assert np.abs(u - u_ref).max() < 2e-5
    for a in u:
        assert np.abs(a.T @ a - np.eye(4)).max() < 1e-5  # expm of an antisymmetric generator
    loss, g = attn.attn_mlp_loss_grad(m, x, ut)
    loss_ref, g_ref = omlp.loss_and_grad(p32, x, ut)
    assert abs(loss - loss_ref) < 1e-5 * max(1.0, loss_ref)
    gr = _flat(g_ref).astype(np.float64)
    assert np.linalg.norm(g - gr) < 1e-4 * np.linalg.norm(gr)
    attn.attn_mlp_destroy(m)
    attn.attn_destroy(ctx)


def test_training_reduces_loss_like_oracle():
    attn, ctx = lib_and_ctx()
    rng = np.random.default_rng(5)
    p = omlp.init_params(1)
    x, ut = _batch(rng, 32)
    m = attn.attn_mlp_create(ctx, _flat(p))
    l0, _ = attn.attn_mlp_loss_grad(m, x, ut)
    l1 = attn.attn_mlp_train(m, x, ut, 60, 3e-3)
    # the FP64 oracle's Adam on the same data and schedule
    q = _unflat(_flat(p))
    opt = omlp.Adam(q, lr=3e-3)
    for _ in range(60):
        lr_, g = omlp.loss_and_grad(q, x, ut)
        opt.step(q, g)
    lref, _ = omlp.loss_and_grad(q, x, ut)
    assert l1 < 0.5 * l0
    assert abs(l1 - lr_) < 1e-2 * l0  # same trajectory up to FP32 rounding
    attn.attn_mlp_destroy(m)
    attn.attn_destroy(ctx)


def test_adam_steps_match_oracle_per_parameter():
    """Three Adam steps of the GPU kernel against the oracle's Adam fed with the same
    FP32 gradients (read back before each step) and the kernel's FP32 constants:
    every parameter agrees to FP32 rounding (3e-7 relative to the parameter plus
    5e-5 of the step size, the bias corrections 1 - b^t being formed in FP32)."""
    attn, ctx = lib_and_ctx()
    rng = np.random.default_rng(9)
    p = omlp.init_params(2)
    x, ut = _batch(rng, 16)
    lr = 1e-3
    m = attn.attn_mlp_create(ctx, _flat(p))
    q = _unflat(_flat(p))
    f32 = lambda a: float(np.float32(a))
    opt = omlp.Adam(q, lr=f32(lr), b1=f32(0.9), b2=f32(0.999), eps=f32(1e-8))
    for _ in range(3):
        _, g = attn.attn_mlp_loss_grad(m, x, ut)  # the gradient the next training step uses
        opt.step(q, _unflat(g))
        attn.attn_mlp_train(m, x, ut, 1, lr)
        got = attn.attn_mlp_get_params(m).astype(np.float64)
        ref = np.concatenate([q[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
        # the kernel stores parameters in FP32 after every step (half an ulp each)
        assert np.all(np.abs(got - ref) <= 3e-7 * np.abs(ref) + 5e-5 * lr), np.abs(got - ref).max()
    attn.attn_mlp_destroy(m)
    attn.attn_destroy(ctx)


def _plain_run(attn, ctx, seed, L=8, m=16, sweeps=3, learned=None, max_iter=None):
    tree = Tree(L * L, m)
    model = attn.attn_model_tfim(ctx, L, 3.04)
    st = attn.attn_state_create(ctx, model, m, raw_tree_tensors(tree.shape, seed))
    n = attn.attn_de_place(st, L * L // 4)
    if learned is not None:
        attn.attn_set_learned_init(st, learned)
    cfg = attn.attn_get_config(ctx)
    cfg.de_max_iter = 20 if max_iter is None else max_iter
    attn.attn_set_config(ctx, cfg)
    es = [attn.attn_sweep(st) for _ in range(sweeps)]
    return st, model, n, es


def test_learned_start_gain_over_identity():
    """Train on the disentanglers of plain 8x8 (seeds 0-3) and 16x16 (seeds 0-1)
    TFIM runs (the pairs are the two-site density matrix at the first update and
    the final disentangler), then compare starts on held-out seed-7 runs of both
    sizes before any MERA step (de_max_iter = 0: the first update reports E_k of
    the start). The plain method judges every prediction: it is used only where it
    does not raise E_k. The trained network must be used for some disentanglers
    and lower sum_k E_k strictly."""
    attn, ctx = lib_and_ctx()
    rhos, targets = [], []
    for L, seeds in ((8, range(4)), (16, range(2))):
        for seed in seeds:
            st, model, n, _ = _plain_run(attn, ctx, seed, L=L)
            r, u = attn.attn_de_training_pairs(st, n)
            rhos.append(r)
            targets.append(u)
            attn.attn_state_destroy(st)
            attn.attn_model_destroy(model)
    rho = np.concatenate(rhos)
    ut = np.concatenate(targets)
    m = attn.attn_mlp_create(ctx, _flat(omlp.init_params(0)))
    l0, _ = attn.attn_mlp_loss_grad(m, rho, ut)
    loss = attn.attn_mlp_train(m, rho, ut, 600, 2e-3)
    assert np.isfinite(loss) and loss < l0
    used_total, gain_total = 0, 0.0
    for L in (8, 16):
        res = {}
        for name, lm in (("plain", None), ("learned", m)):
            st, model, n, _ = _plain_run(attn, ctx, 7, L=L, sweeps=2, learned=lm, max_iter=0)
            res[name] = attn.attn_de_energies(st, n)[:, 0]
            if lm is not None:
                used, fb = attn.attn_learned_init_report(st)
                assert used + fb == n
                used_total += used
            attn.attn_state_destroy(st)
            attn.attn_model_destroy(model)
        # the plain method's judgement: a prediction never raises E_k above the plain start
        assert np.all(res["learned"] <= res["plain"] + 1e-12)
        gain = float(np.sum(res["plain"] - res["learned"]))
        print(f"L={L}: learned-start gain in sum_k E_k at the first update {gain:.6e} (used {used} of {n})")
        gain_total += gain
    assert used_total > 0
    assert gain_total > 0.0
    cfg = attn.attn_get_config(ctx)
    cfg.de_max_iter = 20
    attn.attn_set_config(ctx, cfg)
    attn.attn_mlp_destroy(m)
    attn.attn_destroy(ctx)
