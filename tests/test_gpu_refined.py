"""Parity of the refined mixed-precision forms with the FP64 oracle.

The local eigenproblem of Sec. 4.4.2 solved by BF16 Lanczos on the tensor
cores followed by the FP64 Rayleigh-Ritz refinement (Jacobi-Davidson
corrections from BF16 conjugate-gradient solves), with the FP64 contractions
either on FP64 FMAs or as exact BF16 slice products (f64_split), must reach
the oracle's FP64 ground state of the same H_eff within 1e-8 per site; a
whole aTTN run (Sec. 4: disentangler update, mapping, TTN sweep) in that
precision must track the oracle's FP64 run within 1e-8 per site and stay
above the exact ground-state energy.
"""
import numpy as np
import pytest

from inputs import normal, raw_tree_tensors
from oracle.disentangle import map_terms, place_disentanglers, products_of
from oracle.lattice import ground_energy_ed, square_lattice, tfim_terms
from oracle.sweep import attn_ground_state
from oracle.tree import Tree
from oracle.ttn import TTNState
from tests.gpu_util import dev, host, lib_and_ctx

pytestmark = pytest.mark.gpu

MIXED = {"matvec_dtype": 3}  # ATTN_BF16 Lanczos; refinement at the library defaults


def _orthogonal(seed, k):
    q, r = np.linalg.qr(normal(seed, 7000 + k, 16).reshape(4, 4))
    return q * np.sign(np.diag(r))


_LOWEST = {}


def _oracle_lowest(ost, node):
    """Converged lowest eigenpair of the oracle's H_eff at `node`: the oracle applies
    H_eff term by term (its definition) and ARPACK's implicitly restarted Lanczos
    (scipy eigsh, a library step) converges the lowest eigenvalue."""
    import scipy.sparse.linalg as sla

    terms = ost.heff_terms(node)
    shape = ost.T[node].shape

    def apply(x):
        return ost.heff_apply(node, x.reshape(shape), terms)

    op = sla.LinearOperator((ost.T[node].size,) * 2, matvec=lambda v: apply(v).reshape(-1), dtype=np.float64)
    w, v = sla.eigsh(op, k=1, which="SA", v0=ost.T[node].reshape(-1), tol=1e-14)
    lam = float(w[0])
    assert np.linalg.norm(apply(v[:, 0]).reshape(-1) - lam * v[:, 0]) < 1e-10 * abs(lam)
    return lam, apply


@pytest.mark.parametrize("L,m,n_de,split", [(4, 16, 4, 0), (4, 16, 4, 1), (8, 32, 16, 0), (8, 32, 16, 1)])
def test_refined_local_solve_reaches_oracle_ground_state(L, m, n_de, split):
    """Top node of a TFIM aTTN (h = 3.04) with seeded orthogonal disentanglers:
    two consecutive mixed-precision solves (the second starts from the first's
    vector, as the next sweep would) reach the oracle's converged eigenvalue
    within 1e-8 per site; the returned value is the FP64 Rayleigh quotient of the
    returned vector under the oracle's H_eff, and is variational."""
    n = L * L
    lat = square_lattice(L)
    terms = tfim_terms(lat, 3.04)
    tree = Tree(n, m)
    des = place_disentanglers(tree, terms, n_de)
    us = [_orthogonal(L, k) for k in range(len(des))]
    raw = raw_tree_tensors(tree.shape, 0)
    ost = TTNState.from_raw(tree, raw, products_of(map_terms(terms, des, us)))
    node = tree.top_nodes()[0]
    key = (L, m, n_de)
    if key not in _LOWEST:  # the oracle's eigenvalue serves both precision arms
        _LOWEST[key] = _oracle_lowest(ost, node)
    lam, apply = _LOWEST[key]

    attn, ctx = lib_and_ctx(dict(MIXED, f64_split=split))
    mod = attn.attn_model_tfim(ctx, L, 3.04)
    st = attn.attn_state_create(ctx, mod, m, raw)
    assert attn.attn_de_place(st, n_de) == len(des)
    for k, u in enumerate(us):
        attn.attn_de_set(st, k, u)
    attn.attn_map_hamiltonian(st)
    attn.attn_move_centre(st, node)
    H = attn.attn_heff_build(st, node)
    t = dev(attn.attn_node_get(st, node))
    th1, _ = attn.attn_eigsolve(H, t)
    th2, _ = attn.attn_eigsolve(H, t)
    v = host(t)
    rq = float(np.vdot(v, apply(v).reshape(v.shape)) / np.vdot(v, v))
    assert abs(th2 - rq) <= 1e-12 * abs(rq), (th2, rq)
    assert th1 >= lam - 1e-12 * abs(lam) and th2 >= lam - 1e-12 * abs(lam)
    assert abs(th2 - lam) <= 1e-8 * n, (th2, lam, (th2 - lam) / n)
    attn.attn_heff_destroy(H)
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(mod)
    attn.attn_destroy(ctx)


@pytest.mark.parametrize("split", [0, 1])
def test_refined_attn_run_tracks_oracle(split):
    """4x4 TFIM (h = 3), m = 16, 4 disentanglers, S_TTN = 1, four aTTN sweeps:
    BF16 Lanczos with FP64 refinement on the [16,16,16] top nodes (the smaller
    nodes run FP64) against the oracle's FP64 run from the same raw tensors.
    Both sides use Krylov depth 60, enough for every local problem of this tree to
    converge from its start: a depth-20 FP64 Lanczos stops short of the local
    minimum in the first sweep, which the refined solve then passes (a different
    trajectory, not a different arithmetic)."""
    L, m, n_de = 4, 16, 4
    n = L * L
    lat = square_lattice(L)
    terms = tfim_terms(lat, 3.0)
    tree = Tree(n, m)
    des = place_disentanglers(tree, terms, n_de)
    raw = raw_tree_tensors(tree.shape, 0)
    if "run" not in _LOWEST:  # the oracle's run serves both precision arms
        _LOWEST["run"] = (attn_ground_state(TTNState.from_raw(tree, raw), terms, des, 4, depth=60)[0],
                          ground_energy_ed(n, terms))
    e_ref, e0 = _LOWEST["run"]

    attn, ctx = lib_and_ctx(dict(MIXED, f64_split=split, lanczos_depth=60))
    mod = attn.attn_model_tfim(ctx, L, 3.0)
    st = attn.attn_state_create(ctx, mod, m, raw)
    assert attn.attn_de_place(st, n_de) == len(des)
    e_gpu = [attn.attn_sweep(st) for _ in range(4)]
    for s, (a, b) in enumerate(zip(e_gpu, e_ref)):
        assert abs(a - b) <= 1e-8 * n, (s, a, b, (a - b) / n)
        assert a >= e0 - 1e-9 * abs(e0)
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(mod)
    attn.attn_destroy(ctx)
