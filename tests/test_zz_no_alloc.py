"""The allocation-free H_eff entry point (for callers that cannot allocate
device memory, e.g. under a host framework that owns all free memory or in
code that must not pay cudaFree's device synchronisation) against the regular
entry point, through the C ABI. Collected last on purpose."""
import numpy as np
import pytest

from inputs import random_operators, random_vector
from tests.gpu_util import dev, host, lib_and_ctx, rel_err

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12  # the FP64 H_eff tolerance used by the other parity tests
KINDS = {0: (0, 1), 1: (0, 2), 2: (1, 2)}


def _ops(shape, counts, ntrip, seed):
    h = [dev(random_operators(1, m, seed, 10 + s)[0]) for s, m in enumerate(shape)]
    pairs = {k: (dev(random_operators(counts[k], shape[p], seed, 20 + 2 * k)),
                 dev(random_operators(counts[k], shape[q], seed, 21 + 2 * k)))
             for k, (p, q) in KINDS.items() if counts[k]}
    trip = tuple(dev(random_operators(ntrip, shape[s], seed, 40 + s)) for s in range(3)) if ntrip else None
    return h, pairs, trip


@pytest.mark.parametrize("shape,counts,ntrip", [((5, 7, 6), (4, 3, 2), 2), ((64, 48, 80), (9, 7, 5), 3),
                                                ((128, 128, 128), (6, 4, 4), 0)])
def test_static_scratch_apply_matches_regular_apply(shape, counts, ntrip):
    import torch

    attn, ctx = lib_and_ctx()
    h, pairs, trip = _ops(shape, counts, ntrip, seed=13)
    H = attn.attn_heff_create(ctx, shape, h, pairs, trip)
    for call in range(2):  # two calls in a row share the static scratch
        x = dev(random_vector(shape, 100 + call))
        y_ref = torch.empty_like(x)
        attn.attn_heff_apply(H, x, y_ref, attn.ATTN_F64)
        y = torch.full_like(x, float("nan"))
        attn.attn_heff_apply_f64_static(shape, x, y, h, pairs, trip)
        assert rel_err(host(y), host(y_ref)) < TOL_F64, call
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def test_static_scratch_rejects_oversized_tensors():
    attn, ctx = lib_and_ctx()
    import torch

    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    y = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(attn.AttnError) as e:
        attn.attn_heff_apply_f64_static((256, 128, 128), x, y)  # 4M entries > 2M scratch doubles
    assert e.value.status == 1 and "scratch" in str(e.value)
    attn.attn_destroy(ctx)
