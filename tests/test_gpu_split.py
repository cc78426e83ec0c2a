"""FP64 contractions as exact BF16 slice products (Ozaki scheme) against the oracle.

With ``f64_split`` set, the larger FP64 contractions of an H_eff application
(the per-product mode products and the product-summing stage) run on the tensor
cores from six BF16 slices (7 + 5 x 8 = 47 bits) of every operand row:
  * integer inputs in [-7, 7] keep every intermediate below 2^23, so the first
    three slices hold them exactly, every kept slice product is exact and the
    fixed-point sum is exact: the result equals the oracle's (exact) integer
    arithmetic bit for bit;
  * random inputs meet the FP64 path's tolerance (1e-12 relative, max-abs error
    over max-abs output): the error is about K 2^-46 of the row scales in the
    worst case and a few 2^-46 sqrt(K) in practice.
"""
import numpy as np
import pytest

from inputs import random_operators, random_vector
from inputs.synth import normal
from oracle.ttn import heff_apply_ops, heff_sample_ops
from tests.gpu_util import dev, host, lib_and_ctx, rel_err

pytestmark = pytest.mark.gpu

KINDS = {0: (0, 1), 1: (0, 2), 2: (1, 2)}


def _ints(count, dim, seed, stream):
    """Random integer matrices with entries in [-7, 7] (symmetric, like link operators)."""
    g = np.rint(normal(seed, stream, count * dim * dim).reshape(count, dim, dim) * 2.5)
    g = np.clip(np.rint((g + g.transpose(0, 2, 1)) / 2), -7, 7)
    return g


def _apply(attn, ctx, shape, h, pairs, trip, x, dtype):
    import torch
    H = attn.attn_heff_create(ctx, shape, [dev(a) if a is not None else None for a in h],
                              {k: (dev(a), dev(b)) for k, (a, b) in pairs.items()},
                              tuple(dev(t) for t in trip) if trip is not None else None)
    xd = dev(x)
    yd = torch.full_like(xd, float("nan"))
    attn.attn_heff_apply(H, xd, yd, dtype)
    attn.attn_sync(ctx)
    y = host(yd)
    attn.attn_heff_destroy(H)
    return y


def test_split_heff_is_exact_on_small_integers():
    shape, counts, nt = (128, 128, 128), (4, 2, 2), 2
    h = tuple(_ints(1, m, 3, 10 + s)[0] for s, m in enumerate(shape))
    pairs = {k: (_ints(counts[k], shape[p], 3, 20 + 2 * k), _ints(counts[k], shape[q], 3, 21 + 2 * k))
             for k, (p, q) in KINDS.items()}
    trip = tuple(_ints(nt, m, 3, 40 + s) for s, m in enumerate(shape))
    x = np.clip(np.rint(random_vector(shape, 5) * 2.5), -7, 7)
    y_ref = heff_apply_ops(x, h, {KINDS[k]: v for k, v in pairs.items()}, trip)
    assert np.abs(y_ref).max() < 2.0 ** 52  # the oracle's FP64 sums are exact integers
    attn, ctx = lib_and_ctx({"f64_split": 1})
    y = _apply(attn, ctx, shape, h, pairs, trip, x, attn.ATTN_F64)
    assert np.array_equal(y, y_ref), float(np.abs(y - y_ref).max())
    attn.attn_destroy(ctx)


@pytest.mark.parametrize("shape,counts,nt", [
    ((64, 64, 64), (40, 20, 20), 3),
    ((100, 72, 130), (30, 20, 20), 2),   # ragged rows and K (padded to 64-wide blocks)
    ((128, 128, 128), (12, 6, 6), 2),
])
def test_split_heff_matches_oracle(shape, counts, nt):
    h = tuple(random_operators(1, m, 7, 10 + s)[0] for s, m in enumerate(shape))
    pairs = {k: (random_operators(counts[k], shape[p], 7, 20 + 2 * k),
                 random_operators(counts[k], shape[q], 7, 21 + 2 * k))
             for k, (p, q) in KINDS.items() if counts[k]}
    trip = tuple(random_operators(nt, m, 7, 40 + s) for s, m in enumerate(shape))
    x = random_vector(shape, 9)
    y_ref = heff_apply_ops(x, h, {KINDS[k]: v for k, v in pairs.items()}, trip)
    attn, ctx = lib_and_ctx({"f64_split": 1})
    y = _apply(attn, ctx, shape, h, pairs, trip, x, attn.ATTN_F64)
    attn.attn_destroy(ctx)
    assert np.isfinite(y).all()
    assert rel_err(y, y_ref) < 1e-12
    # the FP64-FMA path on the same inputs
    attn, ctx = lib_and_ctx()
    y64 = _apply(attn, ctx, shape, h, pairs, trip, x, attn.ATTN_F64)
    attn.attn_destroy(ctx)
    assert rel_err(y, y64) < 1e-12


def test_split_heff_zero_operator_rows_and_slices():
    """Rows of zeros (exponent sentinel) in operators and in x give exact zeros where the
    oracle has them and parity elsewhere."""
    shape, counts = (64, 64, 64), (24, 12, 12)
    pairs = {k: (random_operators(counts[k], shape[p], 8, 20 + 2 * k),
                 random_operators(counts[k], shape[q], 8, 21 + 2 * k)) for k, (p, q) in KINDS.items()}
    for k in pairs:
        a, b = pairs[k]
        a[:, 5, :] = 0.0
        a[:, :, 5] = 0.0
        b[0] = 0.0
    x = random_vector(shape, 4)
    x[:, :, 7] = 0.0
    x[3] = 0.0
    h = (None, None, None)
    y_ref = heff_apply_ops(x, h, {KINDS[k]: v for k, v in pairs.items()})
    attn, ctx = lib_and_ctx({"f64_split": 1})
    y = _apply(attn, ctx, shape, h, pairs, None, x, attn.ATTN_F64)
    attn.attn_destroy(ctx)
    assert rel_err(y, y_ref) < 1e-12
    assert np.all(y[y_ref == 0.0] == 0.0)


def test_split_heff_full_size_sampled():
    """[128]^3 with the product counts of a 32x32 top node, sampled entries."""
    shape, counts, nt = (128, 128, 128), (120, 60, 60), 20
    h = tuple(random_operators(1, m, 12, 10 + s)[0] for s, m in enumerate(shape))
    pairs = {k: (random_operators(counts[k], shape[p], 12, 20 + 2 * k),
                 random_operators(counts[k], shape[q], 12, 21 + 2 * k)) for k, (p, q) in KINDS.items()}
    trip = tuple(random_operators(nt, m, 12, 40 + s) for s, m in enumerate(shape))
    x = random_vector(shape, 13)
    attn, ctx = lib_and_ctx({"f64_split": 1})
    y = _apply(attn, ctx, shape, h, pairs, trip, x, attn.ATTN_F64)
    attn.attn_destroy(ctx)
    rng = np.random.default_rng(3)
    idx = [tuple(int(v) for v in rng.integers(0, 128, 3)) for _ in range(8)]
    ref = heff_sample_ops(x, idx, h, {KINDS[k]: v for k, v in pairs.items()}, trip)
    got = np.array([y[i] for i in idx])
    assert np.abs(got - ref).max() < 1e-12 * np.abs(y).max()


def test_split_sweep_energy_matches_fp64_fma():
    """One aTTN sweep of an 8x8 TFIM at m = 64 (renormalisation, disentangler
    environments and FP64 Lanczos all through the split GEMM) against the same
    sweep on FP64 FMAs."""
    import torch
    from inputs import raw_tree_tensors

    # [child, child, parent] shapes of the binary tree over 64 sites with m = 64
    cap = lambda e: min(2 ** (2 ** e), 64)
    shapes = []
    for l in range(1, 6):
        cd = 2 if l == 1 else cap(l - 1)
        shapes += [(cd, cd, cap(min(l, 5)))] * (64 >> l)
    raw = raw_tree_tensors(shapes, 0)
    es = []
    for split in (0, 1):
        attn, ctx = lib_and_ctx({"f64_split": split})
        model = attn.attn_model_tfim(ctx, 8, 3.04)
        st = attn.attn_state_create(ctx, model, 64, raw)
        attn.attn_de_place(st, 16)
        e = [attn.attn_sweep(st) for _ in range(2)]
        es.append(e)
        attn.attn_state_destroy(st)
        attn.attn_model_destroy(model)
        attn.attn_destroy(ctx)
    torch.cuda.synchronize()
    for a, b in zip(*es):
        assert abs(a - b) <= 1e-10 * abs(b), (a, b)


def test_split_gemm_exact_at_the_accumulation_bound():
    """Every entry 126 (2^40 + 2^32 + 2^24 + 2^16 + 2^8 + 1) 2^-47 has all six slice
    digits equal to 126, so every slice product is 126^2 = 15876 and each diagonal's
    partial sums reach 97 % of 2^24 within its accumulation window (diagonal 0:
    15876 x 1024 over K = 1024). The contraction y[i] = sum_j A[i][j] x[j] of one
    pair product (B = identity) must then equal the scheme's exact fixed-point
    result bit for bit: diagonals d = 0..4 contribute (d + 1) 15876 K at weight
    2^(8 (4 - d)) units, the finest one (6 15876 K) / 256 units (an integer here),
    one unit being 2^-46. A tensor-core accumulator that lost a bit near 2^24
    would move the top diagonals' sums by whole units at weight up to 2^32."""
    m0, m1, m2 = 1024, 8, 8
    F = 126 * sum(1 << (8 * k) for k in range(6))
    v = F * 2.0 ** -47
    assert F < 2 ** 47 and v == F / 2 ** 47
    A = np.full((1, m0, m0), v)
    B = np.eye(m1)[None]
    x = np.full((m0, m1, m2), v)
    attn, ctx = lib_and_ctx({"f64_split": 1})
    y = _apply(attn, ctx, (m0, m1, m2), (None, None, None), {0: (A, B)}, None, x, attn.ATTN_F64)
    K = m0
    acc = sum((d + 1) * 15876 * K << (8 * (4 - d)) for d in range(5)) + (6 * 15876 * K) // 256
    assert (6 * 15876 * K) % 256 == 0
    expected = float(acc) * 2.0 ** -46
    assert np.all(y == expected), (float(y.min()), float(y.max()), expected)
    attn.attn_destroy(ctx)
