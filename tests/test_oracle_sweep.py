"""Pins of Lanczos, the sweep and the disentangler update (Secs. 4, 4.1, 4.4.2)."""
import numpy as np
import pytest

from inputs import raw_tree_tensors, random_vector
from oracle.lattice import chain, tfim_terms, tfim_chain_exact, ground_energy_ed, energy_dense, apply_op
from oracle.tree import Tree
from oracle.disentangle import products_of, map_terms
from oracle.ttn import TTNState
from oracle.lanczos import lanczos_lowest
from oracle.sweep import ttn_sweep, attn_ground_state, local_step
from oracle.de_update import build_problems, optimise_de


def test_lanczos_matches_dense_eigensolver():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(30, 30))
    A = A + A.T
    lam = np.linalg.eigvalsh(A)
    th, v, info = lanczos_lowest(lambda x: A @ x, rng.normal(size=30), depth=30)
    assert abs(th - lam[0]) < 1e-10
    assert np.linalg.norm(A @ v - th * v) < 1e-8
    th20, _, _ = lanczos_lowest(lambda x: A @ x, rng.normal(size=30), depth=5)
    assert th20 >= lam[0] - 1e-12  # Ritz values bound lambda_min from above


def test_exact_case_reaches_closed_form():
    """m >= 2^(N/2): the 16-site TTN holds any state, so sweeps reach the exact energy."""
    tree = Tree(16, 256)
    terms = tfim_terms(chain(16), 1.0)
    st = TTNState.from_raw(tree, raw_tree_tensors(tree.shape, 3), products_of(terms))
    for _ in range(3):
        e, _ = ttn_sweep(st)
    assert abs(e - tfim_chain_exact(16, 1.0)) < 1e-10


def test_c1_attn_sweeps_monotone_and_variational(c1):
    _, terms, tree, des = c1
    e0 = ground_energy_ed(16, terms)
    st = TTNState.from_raw(tree, raw_tree_tensors(tree.shape, 0))
    es, us = attn_ground_state(st, terms, des, 4)
    assert all(e >= e0 - 1e-9 for e in es)
    assert all(b <= a + 1e-10 for a, b in zip(es[:-1], es[1:]))
    assert all(np.abs(u.T @ u - np.eye(4)).max() < 1e-12 for u in us)
    # the final TTN energy under H' equals the aTTN energy of the dense state
    psi = st.dense()
    mapped = map_terms(terms, des, us)
    assert abs(energy_dense(psi, 16, mapped) - es[-1]) < 1e-9
    assert es[-1] - e0 < 5e-3


def test_local_steps_monotone(c1):
    _, terms, tree, _ = c1
    st = TTNState.from_raw(tree, raw_tree_tensors(tree.shape, 1), products_of(terms))
    prev = st.energy()
    for n in tree.post_order():
        e = local_step(st, n)
        assert e <= prev + 1e-12 * abs(prev)
        prev = e


@pytest.fixture(scope="module")
def de_setup(c1):
    _, terms, tree, des = c1
    st = TTNState.from_raw(tree, raw_tree_tensors(tree.shape, 0), products_of(terms))
    ttn_sweep(st)
    return st, terms, des, build_problems(st, terms, des)


def test_rdms_equal_dense(de_setup):
    st, terms, des, probs = de_setup
    psi = st.dense().reshape([2] * 16)
    for p in probs:
        for (sp, _, _), r in zip(p.terms, p.rho):
            t = np.moveaxis(psi, list(sp), list(range(len(sp)))).reshape(2 ** len(sp), -1)
            assert np.abs(r - t @ t.T).max() < 1e-13


def test_de_update_optimality_and_energy(de_setup):
    st, terms, des, probs = de_setup
    psi = st.dense()
    rng = np.random.default_rng(4)
    for k, p in enumerate(probs):
        u0 = np.linalg.qr(rng.normal(size=(4, 4)))[0]
        g = p.gamma(u0)
        w, s, vt = np.linalg.svd(g)
        u = -(vt.T @ w.T)
        assert abs(np.trace(u @ g) + s.sum()) < 1e-12 * max(1, s.sum())  # Eq. cost function
        # E_k(u) - E_k(1) equals the dense energy change with only u_k switched on
        us = [np.eye(4) for _ in des]
        base = energy_dense(psi, 16, map_terms(terms, des, us))
        us[k] = u
        new = energy_dense(psi, 16, map_terms(terms, des, us))
        assert abs((new - base) - (p.energy(u) - p.energy(np.eye(4)))) < 1e-11
        uo, hist = optimise_de(p, np.eye(4))
        assert all(b <= a + 1e-12 for a, b in zip(hist[:-1], hist[1:]))
        assert np.abs(uo.T @ uo - np.eye(4)).max() < 1e-12


def test_riemannian_de_gradient_and_descent(de_setup):
    """Riemannian disentangler optimisation (Sec. 4.1.2) in the oracle: the Euclidean
    gradient matches central finite differences of E_k along random directions, its
    projection is tangent to O(4) (u^T grad antisymmetric), the iteration keeps u
    orthogonal, never raises E_k, shrinks the Riemannian gradient by more than 20x
    and, from the identity, stops (relative change below 1e-12) at the energy of
    the MERA-like update's fixed point (Sec. 4.1.1) within 1e-8."""
    from oracle.de_update import euclidean_gradient, optimise_de, optimise_de_riemannian, tangent

    probs = de_setup[3]
    rng = np.random.default_rng(3)
    for p in probs:
        u0 = np.linalg.qr(rng.normal(size=(4, 4)))[0]
        g = euclidean_gradient(p, u0)
        for _ in range(3):
            z = rng.normal(size=(4, 4))
            fd = (p.energy(u0 + 1e-6 * z) - p.energy(u0 - 1e-6 * z)) / 2e-6
            assert abs(fd - np.sum(g * z)) < 1e-7 * max(1.0, abs(fd))
        rg = tangent(u0, g)
        a = u0.T @ rg
        assert np.abs(a + a.T).max() < 1e-12
        u, hist = optimise_de_riemannian(p, np.eye(4), max_iter=60)
        assert np.abs(u.T @ u - np.eye(4)).max() < 1e-12
        assert all(b <= a + 1e-12 * max(1.0, abs(a)) for a, b in zip(hist[:-1], hist[1:]))
        g0 = np.linalg.norm(tangent(np.eye(4), euclidean_gradient(p, np.eye(4))))
        g1 = np.linalg.norm(tangent(u, euclidean_gradient(p, u)))
        assert g1 < 5e-2 * g0
        e_mera = optimise_de(p, np.eye(4))[1][-1]
        assert abs(hist[-1] - e_mera) <= 1e-8 * abs(e_mera)
