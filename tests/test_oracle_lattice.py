"""Pins of the oracle's lattice, site order and Hamiltonians (Sec. 6)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import eigsh

from oracle.lattice import (X, Z, IY, chain, hilbert_d2xy, square_lattice, tfim_terms,
                            heisenberg_terms, ground_energy_ed, tfim_chain_exact, apply_terms)


@pytest.mark.parametrize("L", [2, 4, 8, 16, 32])
def test_hilbert_bijective_and_adjacent(L):
    pts = [hilbert_d2xy(L, d) for d in range(L * L)]
    assert len(set(pts)) == L * L
    assert all(0 <= x < L and 0 <= y < L for x, y in pts)
    for a, b in zip(pts[:-1], pts[1:]):
        assert abs(a[0] - b[0]) + abs(a[1] - b[1]) == 1
    # each half of the curve is a contiguous half of the lattice (x < L/2 first)
    assert all(x < L // 2 for x, _ in pts[: L * L // 2])
    assert pts[0] == (0, 0) and pts[-1] == (L - 1, 0)


def test_bond_counts():
    assert len(square_lattice(4).bonds) == 24
    assert len(square_lattice(32).bonds) == 1984
    assert len(square_lattice(16, triangular=True).bonds) == 705


def _kron_hamiltonian(n, terms):
    """Sparse H built with Kronecker products, independent of apply_op."""
    dim = 2 ** n
    H = sp.csr_matrix((dim, dim))
    for sites, op in terms:
        assert list(sites) == sorted(sites)
        # factor the term into one-site pieces by the Pauli basis when needed
        k = len(sites)
        if k == 1:
            pieces = [(1.0, [op])]
        else:
            basis = [np.eye(2), X, IY, Z]
            pieces = []
            for a in range(4):
                for b in range(4):
                    P = np.kron(basis[a], basis[b])
                    c = np.trace(P.T @ op) / np.trace(P.T @ P)
                    if abs(c) > 1e-15:
                        pieces.append((c, [basis[a], basis[b]]))
        for c, ops in pieces:
            mats = [sp.identity(2, format="csr")] * n
            for s, o in zip(sites, ops):
                mats[s] = sp.csr_matrix(o)
            m = mats[0]
            for x in mats[1:]:
                m = sp.kron(m, x, format="csr")
            H = H + c * m
    return H


@pytest.mark.parametrize("model", ["tfim", "heis"])
def test_matrix_free_energy_matches_kron_build(model):
    lat = square_lattice(2, triangular=(model == "heis")) if model == "heis" else square_lattice(4)
    n = lat.n
    terms = tfim_terms(lat, 3.0) if model == "tfim" else heisenberg_terms(lat)
    H = _kron_hamiltonian(n, terms)
    rng = np.random.default_rng(0)
    v = rng.normal(size=2 ** n)
    assert np.allclose(H @ v, apply_terms(v, n, terms), atol=1e-12)
    e_kron = eigsh(H, k=1, which="SA", tol=1e-12)[0][0]
    assert abs(ground_energy_ed(n, terms) - e_kron) < 1e-9


@pytest.mark.parametrize("n,h", [(8, 0.5), (12, 1.0), (16, 3.0)])
def test_ed_matches_free_fermion_chain(n, h):
    terms = tfim_terms(chain(n), h)
    assert abs(ground_energy_ed(n, terms) - tfim_chain_exact(n, h)) < 1e-9


def test_heisenberg_bond_is_spin_dot_spin():
    terms = heisenberg_terms(chain(2))
    H = sum(op for _, op in terms)
    # singlet energy -3/4, triplet +1/4 for S_i . S_j
    assert np.allclose(np.sort(np.linalg.eigvalsh(H)), [-0.75, 0.25, 0.25, 0.25])


def test_tfim_4x4_energy_close_to_critical_value():
    """4x4 OBC ground energy per site is between the pure-field and pure-bond limits."""
    lat = square_lattice(4)
    e = ground_energy_ed(16, tfim_terms(lat, 3.0)) / 16
    assert -3.0 - 24 / 16 < e < -3.0
