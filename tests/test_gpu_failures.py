"""Failure detection without a GPU fault: bad inputs are refused on the host with
the documented status, a tensor-core kernel whose bounded waits give up drains
its copies and reports ATTN_ETIMEOUT (the context stays usable), and an
eigensolve stopped above its tolerance can report ATTN_ENOTCONVERGED."""
import numpy as np
import pytest

from inputs import raw_tree_tensors, random_operators, random_vector
from oracle.tree import Tree
from tests.gpu_util import dev, host, lib_and_ctx

pytestmark = pytest.mark.gpu

ENONFINITE, ENOTISOMETRIC, ENOTCONVERGED, ETIMEOUT = 4, 5, 6, 7


def _status(fn, *a):
    from paper_2507_21236_gb300 import attn

    try:
        fn(*a)
    except attn.AttnError as e:
        return e.status
    return 0


def test_host_inputs_are_validated():
    attn, ctx = lib_and_ctx()
    tree = Tree(16, 8)
    raw = raw_tree_tensors(tree.shape, 0)
    mod = attn.attn_model_tfim(ctx, 4, 3.0)
    bad = [r.copy() for r in raw]
    bad[3].flat[5] = np.nan
    assert _status(attn.attn_state_create, ctx, mod, 8, bad) == ENONFINITE
    st = attn.attn_state_create(ctx, mod, 8, raw)
    t = attn.attn_node_get(st, 2)
    t.flat[0] = np.inf
    assert _status(attn.attn_node_set, st, 2, t) == ENONFINITE
    assert attn.attn_de_place(st, 4) == 4
    u = np.eye(4)
    u[0, 1] = 1e-6  # not orthogonal at the 1e-10 level the call checks
    assert _status(attn.attn_de_set, st, 0, u) == ENOTISOMETRIC
    params = np.zeros(attn.attn_mlp_param_count(), dtype=np.float32)
    params[7] = np.nan
    assert _status(attn.attn_mlp_create, ctx, params) == ENONFINITE
    # the state is untouched by the refused calls
    assert attn.attn_isometry_error(st) < 1e-12
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(mod)
    attn.attn_destroy(ctx)


def _heff(attn, ctx, m=32, npair=12, seed=3):
    h = [dev(random_operators(1, m, seed, 10 + s)[0]) for s in range(3)]
    pairs = {k: (dev(random_operators(npair, m, seed, 20 + k)), dev(random_operators(npair, m, seed, 30 + k)))
             for k in range(3)}
    return attn.attn_heff_create(ctx, (m, m, m), h, pairs, None), (h, pairs)


def test_tensor_core_wait_timeout_is_reported_and_recovers():
    """A consumer-side wait limit of 2 cycles makes every CTA of the tensor-core
    H_eff kernel give up at its first wait: the kernel records the error, stops
    issuing, waits for its issued copies and MMAs, frees tensor memory and returns;
    the eigensolve reports ATTN_ETIMEOUT. With the default limit restored, the same
    context and H_eff apply again as before the failure."""
    import torch

    attn, ctx = lib_and_ctx({"matvec_dtype": 3, "refine_steps": 2})
    H, keep = _heff(attn, ctx)
    x0 = random_vector((32, 32, 32), 5)
    x = dev(x0)
    y64, y_before, y_after = (torch.empty_like(x) for _ in range(3))
    attn.attn_heff_apply(H, x, y64, attn.ATTN_F64)
    attn.attn_heff_apply(H, x, y_before, attn.ATTN_BF16)
    cfg = attn.attn_get_config(ctx)
    cfg.wait_limit_log2 = 1
    attn.attn_set_config(ctx, cfg)
    assert _status(attn.attn_eigsolve, H, dev(x0)) == ETIMEOUT
    cfg.wait_limit_log2 = 0
    attn.attn_set_config(ctx, cfg)
    attn.attn_sync(ctx)  # the error words were read and cleared by the failed call
    attn.attn_heff_apply(H, x, y_after, attn.ATTN_BF16)
    a, b, r = host(y_after), host(y_before), host(y64)
    # FP32 atomics of a split product list may reorder the last bits
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
    assert np.abs(a - r).max() <= 3e-2 * np.abs(r).max()  # BF16 operands, FP32 accumulation
    th, _ = attn.attn_eigsolve(H, dev(x0))
    assert np.isfinite(th)
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def test_unconverged_eigensolve_can_be_reported():
    attn, ctx = lib_and_ctx({"matvec_dtype": 0, "lanczos_depth": 2, "report_unconverged": 1})
    H, keep = _heff(attn, ctx, m=16, npair=4)
    x0 = random_vector((16, 16, 16), 6)
    assert _status(attn.attn_eigsolve, H, dev(x0)) == ENOTCONVERGED
    cfg = attn.attn_get_config(ctx)
    cfg.lanczos_depth = 60
    cfg.lanczos_tol = 1e-3
    attn.attn_set_config(ctx, cfg)
    th, _ = attn.attn_eigsolve(H, dev(x0))  # converges: no error
    cfg.report_unconverged = 0
    cfg.lanczos_depth = 2
    attn.attn_set_config(ctx, cfg)
    th2, _ = attn.attn_eigsolve(H, dev(x0))  # not reported unless asked for
    assert th2 >= th - 1e-12 * abs(th)
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def test_config_fields_are_validated():
    """attn_set_config refuses out-of-range choices with ATTN_EINVAL and keeps the old
    configuration; valid values are accepted."""
    EINVAL = 1
    attn, ctx = lib_and_ctx()
    good = attn.attn_get_config(ctx)
    for field, bad in (("tc_schedule", 3), ("tc_schedule", -1), ("lanczos_basis", 2), ("de_method", 2),
                       ("wait_limit_log2", 63), ("lanczos_depth", 61)):
        cfg = attn.attn_get_config(ctx)
        setattr(cfg, field, bad)
        assert _status(attn.attn_set_config, ctx, cfg) == EINVAL, field
        assert getattr(attn.attn_get_config(ctx), field) == getattr(good, field), field
    for field, ok in (("tc_schedule", 2), ("lanczos_basis", 1)):
        cfg = attn.attn_get_config(ctx)
        setattr(cfg, field, ok)
        attn.attn_set_config(ctx, cfg)
        assert getattr(attn.attn_get_config(ctx), field) == ok
    attn.attn_destroy(ctx)
