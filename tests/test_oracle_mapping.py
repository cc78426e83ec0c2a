"""Pins of disentangler placement and the mapping H' = D^T H D (Secs. 4.3, 6.1)."""
import os

import numpy as np
import pytest

from oracle.lattice import square_lattice, tfim_terms, heisenberg_terms, apply_op, apply_terms
from oracle.tree import Tree
from oracle.disentangle import (place_disentanglers, check_restrictions, map_terms,
                                split_products, reassemble, products_of)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_c1_placement_golden(c1):
    _, _, _, des = c1
    rows = [tuple(map(int, l.split())) for l in open(os.path.join(GOLDEN, "c1_disentanglers.txt"))
            if l.strip() and not l.startswith("#")]
    assert des == rows


@pytest.mark.parametrize("L,m,tri,req", [(8, 32, False, 16), (16, 64, False, 64),
                                         (16, 64, True, 64), (32, 128, False, 256)])
def test_placement_respects_restrictions(L, m, tri, req):
    lat = square_lattice(L, triangular=tri)
    terms = heisenberg_terms(lat) if tri else tfim_terms(lat, 3.04)
    tree = Tree(L * L, m)
    des = place_disentanglers(tree, terms, req)
    assert 0 < len(des) <= req
    assert check_restrictions(tree, terms, des)
    bonds = set(lat.bonds)
    assert all(d in bonds for d in des)  # each lies fully on an interaction term
    # no pair of one bottom tensor (restriction 2 consequence)
    assert all(i // 2 != j // 2 for i, j in des)


def test_restriction_checker_rejects_violations(c1):
    _, terms, tree, des = c1
    assert not check_restrictions(tree, terms, des + [(2, 13)])  # bond (1,2) touches two
    assert not check_restrictions(tree, terms, [(0, 1)])         # same bottom tensor


def _random_orthogonal(rng, n=4):
    q, r = np.linalg.qr(rng.normal(size=(n, n)))
    return q * np.sign(np.diag(r))


def test_mapping_equals_dense_conjugation(c1):
    _, terms, _, des = c1
    rng = np.random.default_rng(7)
    us = [_random_orthogonal(rng) for _ in des]
    mapped = map_terms(terms, des, us)

    def D(p, t=False):
        for (i, j), u in zip(des, us):
            p = apply_op(p, 16, (i, j), u.T if t else u)
        return p

    x = rng.normal(size=2 ** 16)
    lhs = D(apply_terms(D(x), 16, terms), t=True)
    rhs = apply_terms(x, 16, mapped)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()


def test_identity_disentanglers_leave_h_unchanged(c1):
    _, terms, _, des = c1
    mapped = map_terms(terms, des, [np.eye(4)] * len(des))
    rng = np.random.default_rng(3)
    x = rng.normal(size=2 ** 16)
    assert np.allclose(apply_terms(x, 16, mapped), apply_terms(x, 16, terms), atol=1e-12)


def test_products_reassemble_and_bond_bound(c1):
    _, terms, _, des = c1
    rng = np.random.default_rng(11)
    mapped = map_terms(terms, des, [_random_orthogonal(rng) for _ in des])
    for sites, op in mapped:
        pr = split_products(sites, op)
        assert np.allclose(reassemble(sites, pr), op, atol=1e-13)
        if len(sites) == 2:
            assert len(pr) <= 4  # bond dimension <= d^2 (Sec. 4.3)
    # a 3-site term from a 2-body bond and a disentangler keeps rank <= 4 per cut
    three = [(s, o) for s, o in mapped if len(s) == 3]
    assert three and all(len(split_products(s, o)) <= 16 for s, o in three)
