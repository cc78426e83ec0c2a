"""Parity of the CUDA H_eff path (FP64) with the oracle (Sec. 3.3.2, Sec. 4.4.2).

Tolerance: 1e-12 relative per H_eff application in FP64 (max-abs error over
max-abs of the oracle's output)."""
import numpy as np
import pytest

from inputs import random_operators, random_vector
from oracle.ttn import heff_apply_ops, heff_sample_ops
from tests.gpu_util import dev, host, lib_and_ctx, rel_err

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12
KINDS = {0: (0, 1), 1: (0, 2), 2: (1, 2)}


def _random_heff(shape, counts, n_triple, seed, with_hint=True):
    h = tuple(random_operators(1, m, seed, 10 + s)[0] if with_hint else None for s, m in enumerate(shape))
    pairs = {}
    for k, (p, q) in KINDS.items():
        if counts[k]:
            pairs[k] = (random_operators(counts[k], shape[p], seed, 20 + 2 * k),
                        random_operators(counts[k], shape[q], seed, 21 + 2 * k))
    trip = None
    if n_triple:
        trip = tuple(random_operators(n_triple, shape[s], seed, 40 + s) for s in range(3))
    return h, pairs, trip


def _oracle_pairs(pairs):
    return {KINDS[k]: v for k, v in pairs.items()}


@pytest.mark.parametrize("shape,counts,ntrip", [
    ((2, 2, 4), (3, 2, 2), 1),
    ((5, 7, 6), (4, 3, 2), 2),
    ((16, 16, 32), (20, 10, 10), 3),
    ((100, 72, 130), (7, 5, 6), 2),   # ragged, several 64-wide tiles
    ((32, 32, 32), (120, 40, 40), 4),
    ((64, 64, 64), (40, 20, 20), 3),  # product sums split over CTA groups (64 output tiles)
])
def test_explicit_heff_f64_matches_oracle(shape, counts, ntrip):
    attn, ctx = lib_and_ctx()
    h, pairs, trip = _random_heff(shape, counts, ntrip, seed=7)
    x = random_vector(shape, 3)
    y_ref = heff_apply_ops(x, h, _oracle_pairs(pairs), trip)
    hd = [dev(a) if a is not None else None for a in h]
    pd = {k: (dev(a), dev(b)) for k, (a, b) in pairs.items()}
    td = tuple(dev(a) for a in trip) if trip else None
    H = attn.attn_heff_create(ctx, shape, hd, pd, td)
    xd = dev(x)
    import torch
    yd = torch.full_like(xd, float("nan"))  # poisoned output: every element must be written
    attn.attn_heff_apply(H, xd, yd, attn.ATTN_F64)
    y = host(yd)
    assert np.isfinite(y).all()
    assert rel_err(y, y_ref) < TOL_F64
    # host-buffer entry point gives the same result
    assert rel_err(attn.attn_heff_apply_host(H, x), y_ref) < TOL_F64
    npair, nt, flops = attn.attn_heff_info(H)
    assert npair == tuple(counts) and nt == ntrip
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def test_explicit_heff_f64_full_size_sampled():
    """[128,128,128] with 300 products per pair kind, checked on sampled outputs."""
    shape = (128, 128, 128)
    attn, ctx = lib_and_ctx()
    h, pairs, trip = _random_heff(shape, (300, 60, 60), 4, seed=11)
    x = random_vector(shape, 5)
    H = attn.attn_heff_create(ctx, shape, [dev(a) for a in h],
                              {k: (dev(a), dev(b)) for k, (a, b) in pairs.items()}, tuple(dev(a) for a in trip))
    xd = dev(x)
    import torch
    yd = torch.empty_like(xd)
    attn.attn_heff_apply(H, xd, yd, attn.ATTN_F64)
    y = host(yd)
    rng = np.random.default_rng(0)
    idx = [tuple(int(v) for v in rng.integers(0, 128, 3)) for _ in range(24)] + [(0, 0, 0), (127, 127, 127)]
    ref = heff_sample_ops(x, idx, h, _oracle_pairs(pairs), trip)
    got = np.array([y[i] for i in idx])
    assert np.abs(got - ref).max() < TOL_F64 * np.abs(ref).max() * 10
    # Hermiticity at full size: <z, H x> = <H z, x>
    z = random_vector(shape, 6)
    zd = dev(z)
    wd = torch.empty_like(zd)
    attn.attn_heff_apply(H, zd, wd, attn.ATTN_F64)
    a = float(torch.dot(zd.reshape(-1), yd.reshape(-1)))
    b = float(torch.dot(wd.reshape(-1), xd.reshape(-1)))
    assert abs(a - b) < 1e-11 * abs(a)
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def test_explicit_heff_empty_lists():
    """Only internal operators, no products; and no operators at all (y = 0)."""
    shape = (3, 4, 5)
    attn, ctx = lib_and_ctx()
    h, _, _ = _random_heff(shape, (0, 0, 0), 0, seed=2)
    x = random_vector(shape, 1)
    H = attn.attn_heff_create(ctx, shape, [dev(a) for a in h])
    assert rel_err(attn.attn_heff_apply_host(H, x), heff_apply_ops(x, h)) < TOL_F64
    attn.attn_heff_destroy(H)
    H0 = attn.attn_heff_create(ctx, shape)
    assert np.abs(attn.attn_heff_apply_host(H0, x)).max() == 0.0
    attn.attn_heff_destroy(H0)
    attn.attn_destroy(ctx)


def test_invalid_arguments_are_errors():
    attn, ctx = lib_and_ctx()
    with pytest.raises(attn.AttnError):
        attn.attn_heff_create(ctx, (0, 4, 4))
    H = attn.attn_heff_create(ctx, (2, 2, 2))
    x = dev(np.zeros((2, 2, 2)))
    with pytest.raises(attn.AttnError):
        attn.attn_heff_apply(H, x, x)  # aliasing is rejected
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)
