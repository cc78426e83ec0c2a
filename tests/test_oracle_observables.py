"""Pins of the oracle's aTTN observables (Eq. obs, Eq. corrmat) against the dense
16-site state |psi_aTTN> = D |psi_TTN>."""
import numpy as np
import pytest

from inputs import normal, raw_tree_tensors
from oracle.disentangle import place_disentanglers
from oracle.lattice import square_lattice, tfim_terms
from oracle.observables import correlation_matrix, expectation
from oracle.tree import Tree
from oracle.ttn import TTNState

X = np.array([[0.0, 1.0], [1.0, 0.0]])
Z = np.array([[1.0, 0.0], [0.0, -1.0]])
A = np.array([[0.3, -1.2], [0.7, 0.5]])  # a generic real operator (not symmetric)


def _orth(k):
    q, r = np.linalg.qr(normal(3, 900 + k, 16).reshape(4, 4))
    return q * np.sign(np.diag(r))


@pytest.fixture(scope="module")
def setup():
    lat = square_lattice(4)
    terms = tfim_terms(lat, 3.0)
    tree = Tree(16, 8)
    des = place_disentanglers(tree, terms, 4)
    us = [_orth(k) for k in range(len(des))]
    st = TTNState.from_raw(tree, raw_tree_tensors(tree.shape, 2))
    # dense aTTN state: every disentangler applied to its pair of the TTN vector
    psi = st.dense().reshape([2] * 16)
    for (i, j), u in zip(des, us):
        psi = np.tensordot(u.reshape(2, 2, 2, 2), psi, axes=([2, 3], [i, j]))
        psi = np.moveaxis(psi, [0, 1], [i, j])
    return st, des, us, psi


def _dense_value(psi, sites, ops):
    phi = psi
    for s, o in zip(sites, ops):
        phi = np.moveaxis(np.tensordot(o, phi, axes=(1, s)), 0, s)
    return float(np.vdot(psi, phi) / np.vdot(psi, psi))


def test_dense_state_matches_observables(setup):
    st, des, us, psi = setup
    (i0, j0), (i1, j1) = des[0], des[1]
    free = [s for s in range(16) if all(s not in d for d in des)]
    cases = [([i0], [A]), ([j0], [Z]), ([free[0]], [X]), ([i0, j0], [A, X]), ([j0, i0], [A, Z]),
             ([i0, i1], [X, A]), ([j0, free[1]], [Z, A]), ([free[0], free[1]], [A, A.T]),
             ([i0, j1, free[2]], [X, Z, A])]
    for sites, ops in cases:
        assert abs(expectation(st, des, us, sites, ops) - _dense_value(psi, sites, ops)) < 1e-12, sites
    assert abs(expectation(st, des, us, [i0, i1], [np.eye(2), np.eye(2)]) - 1.0) < 1e-13


def test_correlation_matrix_properties(setup):
    st, des, us, psi = setup
    C = correlation_matrix(st, des, us, X, X)
    assert np.abs(C - C.T).max() < 1e-12
    assert np.abs(np.diag(C) - 1.0).max() < 1e-12  # X^2 = 1
    for i, j in ((0, 5), (des[0][0], des[2][1]), (3, 3)):
        ref = _dense_value(psi, [i], [X @ X]) if i == j else _dense_value(psi, [i, j], [X, X])
        assert abs(C[i, j] - ref) < 1e-12
