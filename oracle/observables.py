"""Observables of the aTTN (Sec. 5: Eq. obs, Eq. corrmat).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definition (Eq. obs with the convention |psi_aTTN> = D |psi_TTN> of the
Hamiltonian mapping): <o>_aTTN = <psi_TTN| D^T o D |psi_TTN>. For an observable
o that is a product of one-site operators on the sites S_o, only the
disentanglers touching S_o act: with S the union of S_o and their pairs, and U
the product of those disentanglers embedded on S (they act on disjoint pairs),
    o' = U^T o U   (on S),    <o> = Tr(rho_S o'),
where rho_S is the reduced density matrix of the TTN on S (the matrix-unit
expectation values of ``de_update.rdms``). No splitting into rank-1 products:
the mapped observable is kept as one explicit operator on S.

Correlation matrix (Eq. corrmat): C[i][j] = <o^a_i o^b_j>, the diagonal being
the one-site observable o^a o^b.

Pins: against the dense 16-site state psi_aTTN = D psi_TTN (each disentangler
applied to the dense TTN vector) for one-site, same-disentangler,
two-disentangler and free-site observables; the identity gives 1; a
correlation matrix of o^a = o^b is symmetric with diagonal <o^2>.
"""
import numpy as np

from .de_update import rdms
from .disentangle import embed


def expectation(state, des, us, sites, ops):
    """<o>_aTTN of o = (x)_a ops[a] on the distinct ``sites`` (any order)."""
    owner = {}
    for k, (i, j) in enumerate(des):
        owner[i] = owner[j] = k
    ks = sorted({owner[s] for s in sites if s in owner})
    S = sorted(set(sites) | {x for k in ks for x in des[k]})
    order = np.argsort(sites)
    o_sites = tuple(sites[a] for a in order)
    o = np.array([[1.0]])
    for a in order:
        o = np.kron(o, np.asarray(ops[a], dtype=np.float64))
    o = embed(o, o_sites, tuple(S))
    U = np.eye(2 ** len(S))
    for k in ks:
        U = U @ embed(np.asarray(us[k], dtype=np.float64), tuple(des[k]), tuple(S))
    o_mapped = U.T @ o @ U
    rho = rdms(state, [tuple(S)])[0]
    return float(np.trace(rho @ o_mapped))


def correlation_matrix(state, des, us, oa, ob):
    """C[i][j] = <o^a_i o^b_j> over all sites (Eq. corrmat)."""
    n = state.tree.n_sites
    ab = np.asarray(oa) @ np.asarray(ob)
    C = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                C[i, j] = expectation(state, des, us, [i], [ab])
            else:
                C[i, j] = expectation(state, des, us, [i, j], [oa, ob])
    return C
