"""The remaining calls of the C ABI against the oracle: renormalisation onto a
link (Fig. eff-op), two-site density matrices and disentangler environments
(Sec. 4.1.1), the update of one disentangler, observables and the correlation
matrix (Sec. 5, Eq. obs, Eq. corrmat), save/resume, a caller-provided device
allocator and the eigensolve on host buffers."""
import os

import numpy as np
import pytest

from inputs import normal, raw_tree_tensors
from oracle.de_update import build_problems, rdms
from oracle.disentangle import map_terms, place_disentanglers, products_of
from oracle.lattice import square_lattice, tfim_terms
from oracle.observables import correlation_matrix, expectation
from oracle.sweep import ttn_sweep
from oracle.tree import Tree
from oracle.ttn import TTNState
from tests.gpu_util import dev, host, lib_and_ctx

pytestmark = pytest.mark.gpu

X = np.array([[0.0, 1.0], [1.0, 0.0]])
Z = np.array([[1.0, 0.0], [0.0, -1.0]])
A = np.array([[0.3, -1.2], [0.7, 0.5]])


def _orth(seed, k):
    q, r = np.linalg.qr(normal(seed, 900 + k, 16).reshape(4, 4))
    return q * np.sign(np.diag(r))


def _pair(L, m, n_de, seed=2, h=3.0, sweep=False, cfg=None):
    """GPU state and oracle state from the same raw tensors and seeded disentanglers
    (optionally after one TTN sweep under the mapped Hamiltonian on both sides)."""
    lat = square_lattice(L)
    terms = tfim_terms(lat, h)
    tree = Tree(L * L, m)
    des = place_disentanglers(tree, terms, n_de)
    us = [_orth(seed, k) for k in range(len(des))]
    raw = raw_tree_tensors(tree.shape, seed)
    ost = TTNState.from_raw(tree, raw, products_of(map_terms(terms, des, us)))
    attn, ctx = lib_and_ctx(cfg)
    mod = attn.attn_model_tfim(ctx, L, h)
    st = attn.attn_state_create(ctx, mod, m, raw)
    assert attn.attn_de_place(st, n_de) == len(des)
    for k, u in enumerate(us):
        attn.attn_de_set(st, k, u)
    attn.attn_map_hamiltonian(st)
    if sweep:
        attn.attn_ttn_sweep(st)
        ttn_sweep(ost)
    return attn, ctx, mod, st, ost, terms, tree, des, us


def _close(attn, ctx, mod, st):
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(mod)
    attn.attn_destroy(ctx)


@pytest.mark.parametrize("L,m,n_de", [(4, 8, 4), (8, 16, 16)])
def test_renormalised_link_operators_match_oracle(L, m, n_de):
    """attn_renormalise moves the centre across a link and renormalises onto it; the
    internal (summed) operator of every product behind the link equals the oracle's
    sum of its per-product renormalised operators, and the open count agrees."""
    attn, ctx, mod, st, ost, terms, tree, des, us = _pair(L, m, n_de)
    for node in (tree.top_nodes()[0], tree.node_id(2, 1), tree.node_id(tree.nL - 1, 0)):
        for slot in (0, 1, 2):
            kind, nb, back = tree.nbr[node][slot]
            if kind != "node":
                continue
            n_open = attn.attn_renormalise(st, node, slot)
            ost.move_centre(nb)
            ops = ost.link_ops(nb, back)
            region = set(tree.region(nb, back))
            internal = [q for q in ops if set(ost.products[q][0]) <= region]
            ref = sum((ops[q] for q in internal), np.zeros((tree.shape[nb][back],) * 2))
            d, n2, has, h = attn.attn_link_operators(st, nb, back)
            assert n2 == n_open == len(ops) - len(internal)
            assert has == bool(internal)
            assert np.abs(h - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (node, slot)
    _close(attn, ctx, mod, st)


@pytest.mark.parametrize("L,m,n_de,sweep", [(4, 8, 4, True), (8, 16, 16, False)])
def test_rdm2_and_environments_match_oracle(L, m, n_de, sweep):
    """Two-site density matrices of the TTN on every disentangler and Gamma_k, E_k at
    a given u (Eq. contracted) agree with the oracle's RDM route to 1e-12."""
    attn, ctx, mod, st, ost, terms, tree, des, us = _pair(L, m, n_de, sweep=sweep)
    probs = build_problems(ost, terms, des)
    ref_rho = rdms(ost, [tuple(d) for d in des])
    for k in range(len(des)):
        rho = attn.attn_rdm2(st, k)
        assert np.abs(rho - ref_rho[k]).max() <= 1e-12, k
        assert abs(np.trace(rho) - 1.0) < 1e-12
        for u in (np.eye(4), _orth(11, k)):
            g, e = attn.attn_de_environment(st, k, u)
            gr = probs[k].gamma(u)
            assert np.abs(g - gr).max() <= 1e-12 * max(1.0, np.abs(gr).max()), k
            er = probs[k].energy(u)
            assert abs(e - er) <= 1e-12 * max(1.0, abs(er)), k
    _close(attn, ctx, mod, st)


def test_single_disentangler_update():
    """Updating disentangler k alone changes u_k only, and reaches the same u_k and E_k
    as the batched update from the same state."""
    out = {}
    for mode in ("one", "all"):
        attn, ctx, mod, st, ost, terms, tree, des, us = _pair(4, 8, 4, sweep=True)
        if mode == "one":
            before = [attn.attn_de_get(st, k) for k in range(len(des))]
            attn.attn_de_update_one(st, 2)
            after = [attn.attn_de_get(st, k) for k in range(len(des))]
            for k in range(len(des)):
                if k != 2:
                    assert np.array_equal(before[k], after[k])
        else:
            attn.attn_de_update(st)
        out[mode] = (attn.attn_de_get(st, 2), attn.attn_de_energies(st, len(des))[2])
        _close(attn, ctx, mod, st)
    assert np.abs(out["one"][0] - out["all"][0]).max() < 1e-10
    assert np.abs(out["one"][1] - out["all"][1]).max() < 1e-12 * np.abs(out["all"][1]).max()


@pytest.mark.parametrize("L,m,n_de,sweep", [(4, 8, 4, True), (8, 16, 16, False)])
def test_observables_match_oracle(L, m, n_de, sweep):
    attn, ctx, mod, st, ost, terms, tree, des, us = _pair(L, m, n_de, sweep=sweep)
    n = L * L
    (i0, j0), (i1, j1) = des[0], des[1]
    free = [s for s in range(n) if all(s not in d for d in des)]
    cases = [([i0], [A]), ([free[0]], [X]), ([i0, j0], [A, X]), ([j0, i0], [A, Z]), ([i0, i1], [X, A]),
             ([j0, free[1]], [Z, A]), ([free[0], free[-1]], [A, A.T]), ([i0, j1, free[2]], [X, Z, A])]
    vals = attn.attn_measure(st, cases)
    for (sites, ops), v in zip(cases, vals):
        ref = expectation(ost, des, us, sites, ops)
        assert abs(v - ref) <= 1e-12 * max(1.0, abs(ref)), sites
    if L == 4:
        C = attn.attn_correlation_matrix(st, Z, X, n)
        Cr = correlation_matrix(ost, des, us, Z, X)
        assert np.abs(C - Cr).max() <= 1e-12
    else:
        C = attn.attn_correlation_matrix(st, X, X, n)
        assert np.abs(C - C.T).max() <= 1e-12 and np.abs(np.diag(C) - 1.0).max() <= 1e-12
        rng = np.random.default_rng(0)
        for i, j in rng.integers(0, n, size=(12, 2)):
            i, j = int(i), int(j)
            ref = expectation(ost, des, us, [i], [X @ X]) if i == j else expectation(ost, des, us, [i, j], [X, X])
            assert abs(C[i, j] - ref) <= 1e-12, (i, j)
    _close(attn, ctx, mod, st)


def test_saved_state_resumes_bit_for_bit(tmp_path):
    """Two FP64 aTTN sweeps, save, two more; a fresh state loaded from the file and
    swept twice reproduces the energies and every tensor bit for bit."""
    path = str(tmp_path / "attn_state.bin")
    L, m = 4, 8
    tree = Tree(L * L, m)
    raw = raw_tree_tensors(tree.shape, 0)
    attn, ctx = lib_and_ctx()
    mod = attn.attn_model_tfim(ctx, L, 3.0)
    st = attn.attn_state_create(ctx, mod, m, raw)
    attn.attn_de_place(st, 4)
    attn.attn_sweep(st)
    attn.attn_sweep(st)
    attn.attn_state_save(st, path)
    e_ref = [attn.attn_sweep(st) for _ in range(2)]
    t_ref = [attn.attn_node_get(st, i) for i in range(tree.n_nodes)]
    st2 = attn.attn_state_create(ctx, mod, m, raw_tree_tensors(tree.shape, 5))  # other tensors
    attn.attn_state_load(st2, path)
    e2 = [attn.attn_sweep(st2) for _ in range(2)]
    assert e2 == e_ref
    for i in range(tree.n_nodes):
        assert np.array_equal(attn.attn_node_get(st2, i), t_ref[i])
    # a file of another model is refused
    mod2 = attn.attn_model_tfim(ctx, L, 2.0)
    st3 = attn.attn_state_create(ctx, mod2, m, raw)
    with pytest.raises(attn.AttnError) as e:
        attn.attn_state_load(st3, path)
    assert e.value.status == 1
    for s in (st, st2, st3):
        attn.attn_state_destroy(s)
    attn.attn_model_destroy(mod)
    attn.attn_model_destroy(mod2)
    attn.attn_destroy(ctx)


def test_caller_allocator_owns_device_memory():
    """With PyTorch's caching allocator installed, the library's device memory comes
    from it (torch accounts for it while handles live and gets it all back), and a
    deterministic FP64 sweep gives the same energies as with cudaMalloc."""
    import torch
    from paper_2507_21236_gb300 import attn as A_

    L, m = 4, 8
    tree = Tree(L * L, m)
    raw = raw_tree_tensors(tree.shape, 0)
    energies = {}
    for use_torch in (False, True):
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()
        if use_torch:
            A_.attn_set_allocator(lambda n, d: torch.cuda.caching_allocator_alloc(n, d),
                                  lambda p, n, d: torch.cuda.caching_allocator_delete(p))
        try:
            attn, ctx = lib_and_ctx()
            mod = attn.attn_model_tfim(ctx, L, 3.0)
            st = attn.attn_state_create(ctx, mod, m, raw)
            attn.attn_de_place(st, 4)
            energies[use_torch] = [attn.attn_sweep(st) for _ in range(2)]
            held = torch.cuda.memory_allocated() - base
            if use_torch:
                assert held > 0
            else:
                assert held == 0
            attn.attn_state_destroy(st)
            attn.attn_model_destroy(mod)
            attn.attn_destroy(ctx)
        finally:
            A_.attn_set_allocator(None, None)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    assert energies[True] == energies[False]


def test_eigsolve_on_host_buffers_equals_device_call():
    attn, ctx, mod, st, ost, terms, tree, des, us = _pair(8, 32, 16, cfg={"matvec_dtype": 0})
    node = tree.top_nodes()[0]
    H = attn.attn_heff_build(st, node)
    x0 = attn.attn_node_get(st, node)
    t = dev(x0)
    th_d, it_d = attn.attn_eigsolve(H, t)
    xh = np.ascontiguousarray(x0.copy())
    th_h, it_h = attn.attn_eigsolve_host(H, xh)
    assert th_h == th_d and it_h == it_d
    assert np.array_equal(xh, host(t))
    attn.attn_heff_destroy(H)
    _close(attn, ctx, mod, st)
