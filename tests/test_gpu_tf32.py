"""TF32 tensor-core H_eff (tcgen05 kind::tf32, FP32 accumulation) against the FP64
oracle.

Tolerance, derived from the arithmetic: x and the operators are rounded to TF32
(10 explicit mantissa bits, round to nearest: unit 2^-11, after an FP32 rounding
of 2^-24); the stage-1 result Z_r stays FP32 in tensor memory and the stage-2 MMA
reads its TF32 part (at most 2^-10 relative if the hardware truncates). So every
product term sees at most four roundings of unit u = 2^-10 (six with three-link
products: C_r and W_r = x x_2 C_r too), plus FP32 accumulation over K = Q (stage
1) and R*P (stage 2) terms; componentwise
    |y_tf32 - y| <= ((1+u)^4 - 1 + (Q + R*P + 2) * 2^-24) * y_abs.
The TF32 result must also be clearly closer to FP64 than the BF16 one (u = 2^-8)."""
import numpy as np
import pytest

from inputs import random_operators, random_vector
from oracle.ttn import heff_apply_ops, heff_sample_ops
from tests.gpu_util import dev, host, lib_and_ctx

pytestmark = pytest.mark.gpu

U = 2.0 ** -10
KINDS = {0: (0, 1), 1: (0, 2), 2: (1, 2)}


def _bound(shape, counts, nt=0):
    R = max(counts) + nt + 3
    P = max(shape)
    rounds = 6 if nt else 4
    return (1 + U) ** rounds - 1 + ((2 if nt else 1) * P + R * P + 2) * 2.0 ** -24


def _case(shape, counts, nt, seed):
    h = tuple(random_operators(1, m, seed, 10 + s)[0] for s, m in enumerate(shape))
    pairs = {k: (random_operators(counts[k], shape[p], seed, 20 + 2 * k),
                 random_operators(counts[k], shape[q], seed, 21 + 2 * k))
             for k, (p, q) in KINDS.items() if counts[k]}
    trip = tuple(random_operators(nt, m, seed, 60 + s) for s, m in enumerate(shape)) if nt else None
    return h, pairs, trip


def _apply(attn, ctx, shape, h, pairs, trip, x, dtype, reps=1):
    import torch
    H = attn.attn_heff_create(ctx, shape, [dev(a) for a in h], {k: (dev(a), dev(b)) for k, (a, b) in pairs.items()},
                              tuple(dev(t) for t in trip) if trip is not None else None)
    xd = dev(x)
    yd = torch.full_like(xd, float("nan"))
    for _ in range(reps):  # later calls reuse the built tensor-core state
        attn.attn_heff_apply(H, xd, yd, dtype)
    y = host(yd)
    attn.attn_heff_destroy(H)
    return y


@pytest.mark.parametrize("shape,counts,nt", [
    ((128, 128, 128), (3, 2, 2), 0),
    ((64, 64, 64), (10, 6, 6), 0),
    ((16, 16, 128), (12, 8, 8), 0),
    ((32, 48, 80), (5, 4, 3), 0),      # ragged: partial K blocks, odd slice count
    ((128, 128, 128), (0, 0, 5), 0),   # one kind only
    ((128, 128, 128), (3, 2, 2), 5),   # three-link products beside the pairs
    ((64, 64, 64), (0, 0, 0), 12),     # three-link products only
    ((32, 48, 80), (5, 4, 3), 7),
])
@pytest.mark.parametrize("schedule", [1, 2])  # split grid, persistent (pair products)
def test_tf32_heff_within_rounding_bound(shape, counts, nt, schedule):
    attn, ctx = lib_and_ctx({"tc_schedule": schedule})
    h, pairs, trip = _case(shape, counts, nt, seed=3)
    x = random_vector(shape, 9)
    y = _apply(attn, ctx, shape, h, pairs, trip, x, attn.ATTN_TF32, reps=2)
    yb = _apply(attn, ctx, shape, h, pairs, trip, x, attn.ATTN_BF16)
    op = {KINDS[k]: v for k, v in pairs.items()}
    y64 = heff_apply_ops(x, h, op, trip)
    yabs = heff_apply_ops(np.abs(x), tuple(np.abs(a) for a in h),
                          {k: (np.abs(a), np.abs(b)) for k, (a, b) in op.items()},
                          tuple(np.abs(t) for t in trip) if trip is not None else None)
    assert np.isfinite(y).all()
    b = _bound(shape, counts, nt)
    viol = np.abs(y - y64) - b * yabs
    assert viol.max() <= 1e-30, (float(viol.max()), b)
    e_tf = np.linalg.norm(y - y64) / np.linalg.norm(yabs)
    e_bf = np.linalg.norm(yb - y64) / np.linalg.norm(yabs)
    assert e_tf < U and e_tf < e_bf / 4, (e_tf, e_bf)
    attn.attn_destroy(ctx)


def test_tf32_heff_full_size_sampled():
    """[128]^3 with ~300 products per kind and 100 three-link products (the size of
    the 32x32, m = 128 nodes), sampled entries."""
    shape, counts, nt = (128, 128, 128), (300, 120, 120), 100
    attn, ctx = lib_and_ctx()
    h, pairs, trip = _case(shape, counts, nt, seed=21)
    x = random_vector(shape, 4)
    y = _apply(attn, ctx, shape, h, pairs, trip, x, attn.ATTN_TF32, reps=2)
    op = {KINDS[k]: v for k, v in pairs.items()}
    rng = np.random.default_rng(1)
    idx = [tuple(int(v) for v in rng.integers(0, 128, 3)) for _ in range(8)]
    ref = heff_sample_ops(x, idx, h, op, trip)
    absref = heff_sample_ops(np.abs(x), idx, tuple(np.abs(a) for a in h),
                             {k: (np.abs(a), np.abs(b)) for k, (a, b) in op.items()}, tuple(np.abs(t) for t in trip))
    got = np.array([y[i] for i in idx])
    assert np.all(np.abs(got - ref) <= _bound(shape, counts, nt) * absref)
    attn.attn_destroy(ctx)


def test_tf32_mixed_eigsolve_reaches_fp64_eigenpair():
    """TF32 Lanczos + FP64 Jacobi-Davidson refinement on a physical H_eff (8x8 TFIM,
    m = 32, top node after one sweep) reaches the converged FP64 eigenvalue to 1e-11
    relative, like the BF16 form, with the FP64 Rayleigh quotient returned."""
    import torch
    from inputs import raw_tree_tensors
    from oracle.tree import Tree

    attn, ctx = lib_and_ctx()
    tree = Tree(64, 32)
    model = attn.attn_model_tfim(ctx, 8, 3.04)
    st = attn.attn_state_create(ctx, model, 32, raw_tree_tensors(tree.shape, 0))
    attn.attn_de_place(st, 16)
    attn.attn_map_hamiltonian(st)
    attn.attn_ttn_sweep(st)
    node = tree.top_nodes()[0]
    attn.attn_move_centre(st, node)
    H = attn.attn_heff_build(st, node)
    x0 = attn.attn_node_get(st, node)
    cfg = attn.attn_get_config(ctx)
    cfg.lanczos_depth, cfg.lanczos_tol, cfg.matvec_dtype = 60, 1e-14, attn.ATTN_F64
    attn.attn_set_config(ctx, cfg)
    th64, _ = attn.attn_eigsolve(H, dev(x0))
    cfg.lanczos_depth, cfg.lanczos_tol, cfg.matvec_dtype = 20, 1e-13, attn.ATTN_TF32
    cfg.refine_steps, cfg.refine_tol, cfg.refine_inner = 5, 1e-13, 16
    attn.attn_set_config(ctx, cfg)
    t = dev(x0)
    th, _ = attn.attn_eigsolve(H, t)
    w = torch.empty_like(t)
    attn.attn_heff_apply(H, t, w, attn.ATTN_F64)
    rq = float(torch.dot(t.reshape(-1), w.reshape(-1)) / torch.dot(t.reshape(-1), t.reshape(-1)))
    assert abs(th - rq) < 1e-12 * abs(rq)
    assert th >= th64 - 1e-11 * abs(th64) and th - th64 < 1e-11 * abs(th64), (th, th64)
    attn.attn_heff_destroy(H)
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(model)
    attn.attn_destroy(ctx)
