"""BF16 tensor-core H_eff (tcgen05) against the FP64 oracle.

Tolerance, derived from the arithmetic: every product term sees at most four
BF16 roundings (x, A_r, B_r and the stage-1 result Z_r), each with unit
roundoff u = 2^-8, plus FP32 accumulation over K = Q (stage 1) and R*P
(stage 2) terms. Componentwise,
    |y_bf16 - y| <= ((1+u)^4 - 1 + (Q + R*P + 2) * 2^-24) * y_abs,
with y_abs the same contraction applied to |x| and the entrywise absolute
operators. The test checks that bound elementwise, plus a typical-size check
on the normwise error.
"""
import numpy as np
import pytest

from inputs import random_operators, random_vector
from oracle.ttn import heff_apply_ops, heff_sample_ops
from tests.gpu_util import dev, host, lib_and_ctx

pytestmark = pytest.mark.gpu

U = 2.0 ** -8
KINDS = {0: (0, 1), 1: (0, 2), 2: (1, 2)}


def _bound(shape, counts):
    R = max(counts) + 3
    P = max(shape)
    return (1 + U) ** 4 - 1 + (P + R * P + 2) * 2.0 ** -24


def _case(shape, counts, seed, with_hint=True):
    h = tuple(random_operators(1, m, seed, 10 + s)[0] if with_hint else None for s, m in enumerate(shape))
    pairs = {k: (random_operators(counts[k], shape[p], seed, 20 + 2 * k),
                 random_operators(counts[k], shape[q], seed, 21 + 2 * k))
             for k, (p, q) in KINDS.items() if counts[k]}
    return h, pairs


@pytest.mark.parametrize("schedule", [1, 2])  # split grid, persistent
@pytest.mark.parametrize("shape,counts", [
    ((128, 128, 128), (3, 2, 2)),
    ((64, 64, 64), (10, 6, 6)),
    ((16, 16, 128), (12, 8, 8)),
    ((32, 48, 80), (5, 4, 3)),       # kinds of different P: persistent runs cross kinds
    ((128, 128, 128), (0, 0, 5)),   # one kind only
])
def test_bf16_heff_within_rounding_bound(shape, counts, schedule):
    attn, ctx = lib_and_ctx({"tc_schedule": schedule})
    h, pairs = _case(shape, counts, seed=3)
    x = random_vector(shape, 9)
    H = attn.attn_heff_create(ctx, shape, [dev(a) for a in h], {k: (dev(a), dev(b)) for k, (a, b) in pairs.items()})
    import torch
    xd = dev(x)
    yd = torch.full_like(xd, float("nan"))
    attn.attn_heff_apply(H, xd, yd, attn.ATTN_BF16)
    y = host(yd)
    op = {KINDS[k]: v for k, v in pairs.items()}
    y64 = heff_apply_ops(x, h, op)
    yabs = heff_apply_ops(np.abs(x), tuple(np.abs(a) for a in h),
                          {k: (np.abs(a), np.abs(b)) for k, (a, b) in op.items()})
    assert np.isfinite(y).all()
    b = _bound(shape, counts)
    viol = np.abs(y - y64) - b * yabs
    assert viol.max() <= 1e-30, (float(viol.max()), b)
    # typical error is far below the worst-case bound
    assert np.linalg.norm(y - y64) / np.linalg.norm(yabs) < U
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


@pytest.mark.parametrize("schedule", [0, 1, 2])  # timed choice, split grid, persistent
def test_bf16_heff_full_size_many_products(schedule):
    """[128]^3 with ~300 products per kind (the size of the 32x32, m = 128 top nodes), sampled."""
    shape = (128, 128, 128)
    counts = (300, 120, 120)
    attn, ctx = lib_and_ctx({"tc_schedule": schedule})
    h, pairs = _case(shape, counts, seed=21)
    x = random_vector(shape, 4)
    H = attn.attn_heff_create(ctx, shape, [dev(a) for a in h], {k: (dev(a), dev(b)) for k, (a, b) in pairs.items()})
    import torch
    xd = dev(x)
    yd = torch.empty_like(xd)
    for _ in range(2):  # second call reuses the built tensor-core state
        attn.attn_heff_apply(H, xd, yd, attn.ATTN_BF16)
    y = host(yd)
    op = {KINDS[k]: v for k, v in pairs.items()}
    rng = np.random.default_rng(1)
    idx = [tuple(int(v) for v in rng.integers(0, 128, 3)) for _ in range(16)]
    ref = heff_sample_ops(x, idx, h, op)
    absref = heff_sample_ops(np.abs(x), idx, tuple(np.abs(a) for a in h),
                             {k: (np.abs(a), np.abs(b)) for k, (a, b) in op.items()})
    got = np.array([y[i] for i in idx])
    assert np.all(np.abs(got - ref) <= _bound(shape, counts) * absref)
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def test_bf16_unsupported_shape_is_an_error():
    attn, ctx = lib_and_ctx()
    H = attn.attn_heff_create(ctx, (2, 2, 4))
    import torch
    xd = dev(np.ones((2, 2, 4)))
    yd = torch.empty_like(xd)
    with pytest.raises(attn.AttnError) as e:
        attn.attn_heff_apply(H, xd, yd, attn.ATTN_BF16)
    assert e.value.status == 8
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def test_mixed_precision_eigsolve_is_fp64_accurate():
    """BF16 Lanczos followed by FP64 refinement on a physical H_eff (8x8 TFIM, m = 32,
    top node): the returned value is the FP64 Rayleigh quotient of the returned vector,
    it is variational (>= the converged FP64 eigenvalue) and the refinement lowers the
    FP64 residual of the BF16 Ritz pair (Sec. 4.4.2 with the mixed-precision policy)."""
    from inputs import raw_tree_tensors
    from oracle.tree import Tree

    attn, ctx = lib_and_ctx()
    tree = Tree(64, 32)
    model = attn.attn_model_tfim(ctx, 8, 3.04)
    st = attn.attn_state_create(ctx, model, 32, raw_tree_tensors(tree.shape, 0))
    attn.attn_de_place(st, 16)
    attn.attn_map_hamiltonian(st)
    attn.attn_ttn_sweep(st)  # a physical state
    node = tree.top_nodes()[0]
    attn.attn_move_centre(st, node)
    H = attn.attn_heff_build(st, node)
    x0 = attn.attn_node_get(st, node)
    cfg = attn.attn_get_config(ctx)
    cfg.lanczos_depth = 60
    cfg.lanczos_tol = 1e-14
    cfg.matvec_dtype = attn.ATTN_F64
    attn.attn_set_config(ctx, cfg)
    t64 = dev(x0)
    th64, _ = attn.attn_eigsolve(H, t64)
    import torch

    def rq_and_res(vd):
        w = torch.empty_like(vd)
        attn.attn_heff_apply(H, vd, w, attn.ATTN_F64)
        th = float(torch.dot(vd.reshape(-1), w.reshape(-1)) / torch.dot(vd.reshape(-1), vd.reshape(-1)))
        return th, float(torch.linalg.norm(w - th * vd))

    cfg.lanczos_depth = 20
    cfg.matvec_dtype = attn.ATTN_BF16
    cfg.refine_steps = 0
    attn.attn_set_config(ctx, cfg)
    tlo = dev(x0)
    attn.attn_eigsolve(H, tlo)
    _, res_lo = rq_and_res(tlo)
    cfg.refine_steps = 8
    cfg.refine_tol = 1e-13
    attn.attn_set_config(ctx, cfg)
    tmx = dev(x0)
    thmx, _ = attn.attn_eigsolve(H, tmx)
    rq, res_mx = rq_and_res(tmx)
    assert abs(thmx - rq) < 1e-12 * abs(rq)
    assert thmx >= th64 - 1e-9 * abs(th64)
    assert res_mx < 0.5 * res_lo
    attn.attn_heff_destroy(H)
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(model)
    attn.attn_destroy(ctx)


@pytest.mark.gpu
def test_mixed_precision_refinement_reaches_fp64_eigenpair():
    """Jacobi-Davidson refinement with BF16 inner solves (refine_inner > 0) reaches the
    converged FP64 eigenpair of a physical H_eff (8x8 TFIM, m = 32, top node) within a
    few FP64 matvecs, while the same number of plain residual corrections (refine_inner
    = 0) does not; the returned value is the FP64 Rayleigh quotient of the returned
    vector in both cases (the mixed-precision policy of the local eigenproblem,
    Sec. 4.4.2)."""
    from inputs import raw_tree_tensors
    from oracle.tree import Tree
    import torch

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
    cfg.lanczos_depth = 60
    cfg.lanczos_tol = 1e-14
    cfg.matvec_dtype = attn.ATTN_F64
    attn.attn_set_config(ctx, cfg)
    th64, _ = attn.attn_eigsolve(H, dev(x0))

    def rq_and_res(vd):
        w = torch.empty_like(vd)
        attn.attn_heff_apply(H, vd, w, attn.ATTN_F64)
        th = float(torch.dot(vd.reshape(-1), w.reshape(-1)) / torch.dot(vd.reshape(-1), vd.reshape(-1)))
        return th, float(torch.linalg.norm(w - th * vd))

    out = {}
    for inner in (0, 16):
        cfg.lanczos_depth = 20
        cfg.lanczos_tol = 1e-13
        cfg.matvec_dtype = attn.ATTN_BF16
        cfg.refine_steps = 5
        cfg.refine_tol = 1e-13
        cfg.refine_inner = inner
        attn.attn_set_config(ctx, cfg)
        t = dev(x0)
        th, _ = attn.attn_eigsolve(H, t)
        rq, res = rq_and_res(t)
        assert abs(th - rq) < 1e-12 * abs(rq)
        assert th >= th64 - 1e-11 * abs(th64)
        out[inner] = (th - th64, res)
    # five corrections with BF16 inner solves: FP64-level eigenvalue and eigenvector
    assert out[16][0] < 1e-11 * abs(th64), out
    assert out[16][1] < 1e-6 * abs(th64), out
    # five plain residual corrections leave a clearly larger error
    assert out[0][0] > 10 * out[16][0] and out[0][1] > 10 * out[16][1], out
    attn.attn_heff_destroy(H)
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(model)
    attn.attn_destroy(ctx)


def _bound3(shape, counts, nt):
    """Componentwise bound with three-link products: those terms see six BF16
    roundings (x, C_r, W_r = x x_2 C_r, A_r, B_r, Z_r) and one more FP32 sum
    over K = m2 in the slot-2 contraction."""
    R = max(counts) + nt + 3
    P = max(shape)
    return (1 + U) ** 6 - 1 + (2 * P + R * P + 2) * 2.0 ** -24


@pytest.mark.parametrize("shape,counts,nt", [
    ((128, 128, 128), (3, 2, 2), 5),
    ((64, 64, 64), (0, 0, 0), 12),     # three-link products only
    ((32, 48, 80), (5, 4, 3), 7),      # odd slice count, partial K blocks
    ((16, 16, 128), (6, 0, 4), 9),     # no kind-(0, 2) products
])
def test_bf16_heff_three_link_products_within_rounding_bound(shape, counts, nt):
    attn, ctx = lib_and_ctx()
    h, pairs = _case(shape, counts, seed=5)
    trip = tuple(random_operators(nt, m, 5, 60 + s) for s, m in enumerate(shape))
    x = random_vector(shape, 11)
    H = attn.attn_heff_create(ctx, shape, [dev(a) for a in h], {k: (dev(a), dev(b)) for k, (a, b) in pairs.items()},
                              tuple(dev(t) for t in trip))
    import torch
    xd = dev(x)
    yd = torch.full_like(xd, float("nan"))
    for _ in range(2):  # the second call reuses the built state and must not double-count
        attn.attn_heff_apply(H, xd, yd, attn.ATTN_BF16)
    y = host(yd)
    op = {KINDS[k]: v for k, v in pairs.items()}
    y64 = heff_apply_ops(x, h, op, trip)
    yabs = heff_apply_ops(np.abs(x), tuple(np.abs(a) for a in h),
                          {k: (np.abs(a), np.abs(b)) for k, (a, b) in op.items()}, tuple(np.abs(t) for t in trip))
    assert np.isfinite(y).all()
    b = _bound3(shape, counts, nt)
    viol = np.abs(y - y64) - b * yabs
    assert viol.max() <= 1e-30, (float(viol.max()), b)
    assert np.linalg.norm(y - y64) / np.linalg.norm(yabs) < U
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def test_bf16_heff_three_link_products_full_size_sampled():
    """[128]^3 with 300 three-link products next to the pair products, sampled entries."""
    shape = (128, 128, 128)
    counts, nt = (60, 30, 30), 300
    attn, ctx = lib_and_ctx()
    h, pairs = _case(shape, counts, seed=23)
    trip = tuple(random_operators(nt, m, 23, 60 + s) for s, m in enumerate(shape))
    x = random_vector(shape, 6)
    H = attn.attn_heff_create(ctx, shape, [dev(a) for a in h], {k: (dev(a), dev(b)) for k, (a, b) in pairs.items()},
                              tuple(dev(t) for t in trip))
    import torch
    xd = dev(x)
    yd = torch.empty_like(xd)
    attn.attn_heff_apply(H, xd, yd, attn.ATTN_BF16)
    y = host(yd)
    op = {KINDS[k]: v for k, v in pairs.items()}
    rng = np.random.default_rng(2)
    idx = [tuple(int(v) for v in rng.integers(0, 128, 3)) for _ in range(4)]
    ref = heff_sample_ops(x, idx, h, op, trip)
    absref = heff_sample_ops(np.abs(x), idx, tuple(np.abs(a) for a in h),
                             {k: (np.abs(a), np.abs(b)) for k, (a, b) in op.items()}, tuple(np.abs(t) for t in trip))
    got = np.array([y[i] for i in idx])
    assert np.all(np.abs(got - ref) <= _bound3(shape, counts, nt) * absref)
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def test_bf16_schedules_agree_to_fp32_rounding():
    """The persistent form and the split grid sum the same BF16 products; only the FP32
    summation order differs (where a slice pair's products are split between CTAs the
    partial sums meet by atomics). Each order's FP32 error is at most (R P + Q + 2) 2^-24
    of the summed magnitudes, so at sampled entries the two outputs differ by at most
    twice that, with the magnitudes bounded by the same contraction of |x| and |operators|."""
    import torch
    shape, counts = (128, 128, 128), (290, 290, 290)
    h, pairs = _case(shape, counts, seed=8)
    x = random_vector(shape, 6)
    out = {}
    for schedule in (1, 2):
        attn, ctx = lib_and_ctx({"tc_schedule": schedule})
        H = attn.attn_heff_create(ctx, shape, [dev(a) for a in h], {k: (dev(a), dev(b)) for k, (a, b) in pairs.items()})
        xd = dev(x)
        yd = torch.empty_like(xd)
        attn.attn_heff_apply(H, xd, yd, attn.ATTN_BF16)
        out[schedule] = host(yd)
        attn.attn_heff_destroy(H)
        attn.attn_destroy(ctx)
    op = {KINDS[k]: v for k, v in pairs.items()}
    rng = np.random.default_rng(2)
    idx = [tuple(int(v) for v in rng.integers(0, 128, 3)) for _ in range(16)]
    absref = heff_sample_ops(np.abs(x), idx, tuple(np.abs(a) for a in h),
                             {k: (np.abs(a), np.abs(b)) for k, (a, b) in op.items()})
    R, P = max(counts) + 3, 128
    bound = 2 * (R * P + P + 2) * 2.0 ** -24 * (1 + U) ** 4
    diff = np.array([abs(out[1][i] - out[2][i]) for i in idx])
    assert np.all(diff <= bound * absref), float((diff / absref).max())
    assert np.isfinite(out[2]).all()


@pytest.mark.parametrize("basis", [0, 1])  # FP64, FP32 Krylov basis
def test_refined_eigsolve_with_either_krylov_basis(basis):
    """A BF16 Lanczos with an FP64 or (lanczos_basis = 1) an FP32 Krylov basis and FP32
    reorthogonalisation, followed by five FP64 Jacobi-Davidson corrections with BF16 inner
    solves, reaches the converged FP64 eigenpair of a physical H_eff (8x8 TFIM, m = 32, top
    node) to 1e-11 in theta; the returned value is the FP64 Rayleigh quotient of the
    returned vector. Without refinement both bases give theta to BF16 accuracy."""
    from inputs import raw_tree_tensors
    from oracle.tree import Tree
    import torch

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
    cfg.lanczos_depth, cfg.lanczos_tol, cfg.matvec_dtype = 20, 1e-13, attn.ATTN_BF16
    cfg.lanczos_basis = basis
    cfg.refine_steps = 0
    attn.attn_set_config(ctx, cfg)
    th_lo, _ = attn.attn_eigsolve(H, dev(x0))
    assert abs(th_lo - th64) < 2e-2 * abs(th64)
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
