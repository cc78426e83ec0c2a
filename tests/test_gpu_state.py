"""Parity of the CUDA state path with the oracle: isometrisation and QR moves
(Sec. 3.1), effective operators and H_eff of a node (Sec. 3.3.2), energy,
Lanczos and the TTN sweep (Sec. 4). FP64 throughout; tolerance 1e-12
relative per H_eff application."""
import numpy as np
import pytest

from inputs import raw_tree_tensors, random_vector
from oracle.lattice import square_lattice, tfim_terms, heisenberg_terms, chain, tfim_chain_exact
from oracle.tree import Tree
from oracle.disentangle import place_disentanglers, map_terms, products_of
from oracle.ttn import TTNState
from oracle.sweep import ttn_sweep
from tests.gpu_util import dev, host, lib_and_ctx, rel_err

pytestmark = pytest.mark.gpu


def _random_orthogonal(rng):
    q, r = np.linalg.qr(rng.normal(size=(4, 4)))
    return q * np.sign(np.diag(r))


def _setup(L, m, model, n_de, seed=0, de_seed=5, tri=False):
    lat = square_lattice(L, triangular=tri)
    terms = tfim_terms(lat, 3.0) if model == "tfim" else heisenberg_terms(lat)
    tree = Tree(L * L, m)
    des = place_disentanglers(tree, terms, n_de)
    rng = np.random.default_rng(de_seed)
    us = [_random_orthogonal(rng) for _ in des]
    raw = raw_tree_tensors(tree.shape, seed)
    ost = TTNState.from_raw(tree, raw, products_of(map_terms(terms, des, us)))
    attn, ctx = lib_and_ctx()
    mod = attn.attn_model_tfim(ctx, L, 3.0) if model == "tfim" else attn.attn_model_tri_heisenberg(ctx, L, 1.0)
    st = attn.attn_state_create(ctx, mod, m, raw)
    n = attn.attn_de_place(st, n_de)
    assert attn.attn_de_sites(st, n) == des  # same placement as the oracle's rule
    for k, u in enumerate(us):
        attn.attn_de_set(st, k, u)
    attn.attn_map_hamiltonian(st)
    return attn, ctx, mod, st, ost, tree


def _teardown(attn, ctx, mod, st):
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(mod)
    attn.attn_destroy(ctx)


def test_isometrisation_matches_oracle():
    attn, ctx, mod, st, ost, tree = _setup(4, 8, "tfim", 4)
    for n in range(tree.n_nodes):
        assert rel_err(attn.attn_node_get(st, n), ost.T[n]) < 1e-12
    assert attn.attn_isometry_error(st) < 1e-12
    _teardown(attn, ctx, mod, st)


@pytest.mark.parametrize("L,m,model,n_de,nodes", [
    (4, 8, "tfim", 4, [12, 13, 9, 0, 5]),
    (8, 32, "tfim", 16, [60, 61, 56, 40, 3]),
    (4, 8, "heis", 4, [12, 3, 10]),
])
def test_node_heff_matches_oracle(L, m, model, n_de, nodes):
    attn, ctx, mod, st, ost, tree = _setup(L, m, model, n_de, tri=(model == "heis"))
    import torch
    for node in nodes:
        attn.attn_move_centre(st, node)
        ost.move_centre(node)
        assert rel_err(attn.attn_node_get(st, node), ost.T[node]) < 1e-11
        H = attn.attn_heff_build(st, node)
        x = random_vector(tree.shape[node], node + 1)
        xd = dev(x)
        yd = torch.full_like(xd, float("nan"))
        attn.attn_heff_apply(H, xd, yd, attn.ATTN_F64)
        y_ref = ost.heff_apply_stacked(x, ost.heff_stacked(node))
        assert rel_err(host(yd), y_ref) < 1e-12, node
        attn.attn_heff_destroy(H)
        assert abs(attn.attn_energy(st) - ost.energy()) < 1e-12 * max(1.0, abs(ost.energy())) * 10
    assert attn.attn_isometry_error(st) < 1e-12
    _teardown(attn, ctx, mod, st)


def test_eigsolve_matches_dense():
    attn, ctx, mod, st, ost, tree = _setup(4, 8, "tfim", 4)
    node = 12
    attn.attn_move_centre(st, node)
    ost.move_centre(node)
    H = attn.attn_heff_build(st, node)
    # dense H_eff from the oracle's term list, lowest eigenvalue by a dense eigensolver
    V = int(np.prod(tree.shape[node]))
    stacked = ost.heff_stacked(node)
    cols = [ost.heff_apply_stacked(e.reshape(tree.shape[node]), stacked).reshape(-1) for e in np.eye(V)]
    lam = np.linalg.eigvalsh(np.stack(cols, 1))[0]
    cfg = attn.attn_get_config(ctx)
    cfg.lanczos_depth = 60
    cfg.lanczos_tol = 1e-14
    attn.attn_set_config(ctx, cfg)
    td = dev(ost.T[node])
    theta, iters = attn.attn_eigsolve(H, td)
    assert theta >= lam - 1e-10 and abs(theta - lam) < 1e-9
    v = host(td).reshape(-1)
    Hv = ost.heff_apply_stacked(v.reshape(tree.shape[node]), stacked).reshape(-1)
    assert np.linalg.norm(Hv - theta * v) < 1e-6
    attn.attn_heff_destroy(H)
    _teardown(attn, ctx, mod, st)


def test_ttn_sweep_matches_oracle():
    """One FP64 sweep from identical inputs: same local energies as the oracle."""
    attn, ctx, mod, st, ost, tree = _setup(4, 8, "tfim", 4)
    e_gpu = attn.attn_ttn_sweep(st)
    e_ref, _ = ttn_sweep(ost)
    assert abs(e_gpu - e_ref) < 1e-9
    assert attn.attn_isometry_error(st) < 1e-12
    _teardown(attn, ctx, mod, st)


def test_exact_case_chain16():
    """m = 256 on 16 sites holds any state: GPU sweeps reach the free-fermion energy."""
    attn, ctx = lib_and_ctx()
    terms = tfim_terms(chain(16), 1.0)
    mod = attn.attn_model_terms(ctx, 16, terms)
    tree = Tree(16, 256)
    st = attn.attn_state_create(ctx, mod, 256, raw_tree_tensors(tree.shape, 3))
    attn.attn_de_place(st, 0)
    attn.attn_map_hamiltonian(st)
    for _ in range(3):
        e = attn.attn_ttn_sweep(st)
    assert abs(e - tfim_chain_exact(16, 1.0)) < 1e-10
    _teardown(attn, ctx, mod, st)
