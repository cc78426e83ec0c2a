"""Term compression (Sec. 6.2.2): the mapped terms of H' acting on the same sites
summed into one term before the rank-1 split. The effective Hamiltonian is the
same linear map as the oracle's term-by-term H_eff, with fewer rank-1 products."""
import numpy as np
import pytest

from inputs import raw_tree_tensors, random_vector
from oracle.disentangle import map_terms, place_disentanglers, products_of
from oracle.lattice import heisenberg_terms, square_lattice
from oracle.tree import Tree
from oracle.ttn import TTNState
from tests.gpu_util import dev, host, lib_and_ctx, rel_err

pytestmark = pytest.mark.gpu


def _orth(rng):
    q, r = np.linalg.qr(rng.normal(size=(4, 4)))
    return q * np.sign(np.diag(r))


@pytest.mark.parametrize("L,m,n_de", [(4, 8, 4), (8, 16, 16)])
def test_compressed_heisenberg_heff_matches_oracle(L, m, n_de):
    import torch

    lat = square_lattice(L, triangular=True)
    terms = heisenberg_terms(lat)
    tree = Tree(L * L, m)
    des = place_disentanglers(tree, terms, n_de)
    rng = np.random.default_rng(4)
    us = [_orth(rng) for _ in des]
    raw = raw_tree_tensors(tree.shape, 1)
    counts, energies = {}, {}
    for comp in (0, 1):
        # a fresh oracle state per arm: centre moves change the gauge of the tensors
        ost = TTNState.from_raw(tree, raw, products_of(map_terms(terms, des, us)))
        attn, ctx = lib_and_ctx({"compress_terms": comp})
        mod = attn.attn_model_tri_heisenberg(ctx, L, 1.0)
        st = attn.attn_state_create(ctx, mod, m, raw)
        assert attn.attn_de_place(st, n_de) == len(des)
        for k, u in enumerate(us):
            attn.attn_de_set(st, k, u)
        attn.attn_map_hamiltonian(st)
        counts[comp] = attn.attn_hamiltonian_info(st)
        for node in (tree.top_nodes()[0], tree.node_id(2, 0), tree.node_id(1, 3)):
            attn.attn_move_centre(st, node)
            ost.move_centre(node)
            H = attn.attn_heff_build(st, node)
            x = random_vector(tree.shape[node], node + 7)
            xd = dev(x)
            yd = torch.full_like(xd, float("nan"))
            attn.attn_heff_apply(H, xd, yd, attn.ATTN_F64)
            assert rel_err(host(yd), ost.heff_apply(node, x)) < 1e-12, (comp, node)
            attn.attn_heff_destroy(H)
        energies[comp] = attn.attn_ttn_sweep(st)
        attn.attn_state_destroy(st)
        attn.attn_model_destroy(mod)
        attn.attn_destroy(ctx)
    # three terms per bond (xx, yy, zz) become one wherever they act on the same sites
    assert counts[1][0] < counts[0][0] and counts[1][1] < counts[0][1], counts
    assert abs(energies[1] - energies[0]) <= 1e-10 * abs(energies[0])
