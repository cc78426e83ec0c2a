"""Pins of the TTN state, effective operators and H_eff (Secs. 3.1, 3.3.2, 4.4.2)."""
import numpy as np
import pytest

from inputs import raw_tree_tensors, random_vector, random_operators
from oracle.lattice import apply_terms, energy_dense
from oracle.disentangle import map_terms, products_of
from oracle.ttn import TTNState, heff_apply_ops, heff_sample_ops, mode_product


@pytest.fixture(scope="module")
def mapped_state(c1):
    _, terms, tree, des = c1
    rng = np.random.default_rng(5)
    us = []
    for _ in des:
        q, r = np.linalg.qr(rng.normal(size=(4, 4)))
        us.append(q)
    mapped = map_terms(terms, des, us)
    st = TTNState.from_raw(tree, raw_tree_tensors(tree.shape, 0), products_of(mapped))
    return st, mapped


def test_isometry_after_init_and_moves(mapped_state):
    st, _ = mapped_state
    st = st.copy()
    assert st.isometry_error() < 1e-12
    for target in [0, 9, 13, 5]:
        st.move_centre(target)
        assert st.isometry_error() < 1e-12
        psi = st.dense()
        assert abs(psi @ psi - 1.0) < 1e-12
        assert abs(np.linalg.norm(st.T[target]) - 1.0) < 1e-12  # Fig. iso


@pytest.mark.parametrize("node", [12, 9, 2])
def test_heff_equals_bruteforce_projection(mapped_state, node):
    st, mapped = mapped_state
    st = st.copy()
    st.move_centre(node)
    P = st.embedding(node)
    assert np.abs(P.T @ P - np.eye(P.shape[1])).max() < 1e-12
    x = random_vector(st.T[node].shape, 1)
    y = st.heff_apply(node, x)
    yb = P.T @ apply_terms(P @ x.reshape(-1), 16, mapped)
    assert np.abs(y.reshape(-1) - yb).max() < 1e-13 * np.abs(yb).max()
    # energy identity <T|H_eff|T> = <psi|H'|psi>
    assert abs(st.energy() - energy_dense(st.dense(), 16, mapped)) < 1e-12 * 50
    # hermiticity
    z = random_vector(st.T[node].shape, 2)
    assert abs(np.vdot(z, y) - np.vdot(st.heff_apply(node, z), x)) < 1e-13 * np.abs(y).max() * x.size
    # stacked form is the same map
    assert np.abs(st.heff_apply_stacked(x, st.heff_stacked(node)) - y).max() < 1e-13 * np.abs(y).max()


def test_explicit_ops_apply_and_sampling():
    shape = (5, 7, 6)
    x = random_vector(shape, 3)
    h = tuple(random_operators(1, m, 3, 10 + s)[0] for s, m in enumerate(shape))
    pairs = {(0, 1): (random_operators(4, 5, 3, 20), random_operators(4, 7, 3, 21)),
             (0, 2): (random_operators(3, 5, 3, 22), random_operators(3, 6, 3, 23)),
             (1, 2): (random_operators(2, 7, 3, 24), random_operators(2, 6, 3, 25))}
    triples = (random_operators(2, 5, 3, 26), random_operators(2, 7, 3, 27), random_operators(2, 6, 3, 28))
    y = heff_apply_ops(x, h, pairs, triples)
    # independent dense build: kron of each product (slot 0 most significant)
    V = x.size
    H = np.zeros((V, V))
    I = [np.eye(m) for m in shape]
    for s in range(3):
        mats = list(I)
        mats[s] = h[s]
        H += np.kron(np.kron(mats[0], mats[1]), mats[2])
    for (p, q), (A, B) in pairs.items():
        for r in range(A.shape[0]):
            mats = list(I)
            mats[p], mats[q] = A[r], B[r]
            H += np.kron(np.kron(mats[0], mats[1]), mats[2])
    for r in range(triples[0].shape[0]):
        H += np.kron(np.kron(triples[0][r], triples[1][r]), triples[2][r])
    assert np.abs(H @ x.reshape(-1) - y.reshape(-1)).max() < 1e-12
    idx = [(0, 0, 0), (4, 6, 5), (2, 3, 1)]
    s = heff_sample_ops(x, idx, h, pairs, triples)
    assert np.allclose(s, [y[i] for i in idx], atol=1e-12)
