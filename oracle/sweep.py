"""aTTN ground-state search schedule (Sec. 4, steps 1-3; Sec. 6.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Each sweep: (1) optimise all disentanglers, (2) map H -> H', (3) run a
variational sweep of the TTN under H'. The first ``s_ttn`` = 1 sweeps skip
step (1) (Sec. 6.3: the best schedule runs the first sweep on the TTN only).
Disentanglers start as identities (Sec. 6).

Readings for the TTN sweep (the paper defers to the DMRG literature):
post-order visit (left subtree, right subtree, node), the left top tensor's
half first; the centre moves along the tree path by QR, one hop per link;
at each visited tensor the lowest Ritz pair of H_eff replaces the tensor when
its value does not exceed the current energy (+1e-14 |E|).

Pins: for a 16-site TTN with m >= 256 the sweep reaches the exact ground
energy; every local step is monotone; E >= E_exact throughout.
"""
import numpy as np

from .disentangle import map_terms, products_of
from .de_update import build_problems, optimise_de
from .lanczos import lanczos_lowest


def local_step(state, n, depth=20, tol=1e-13, term_by_term=False):
    """``term_by_term`` applies H_eff one rank-1 product at a time (the definition of
    Sec. 3.3.2) instead of one einsum per slot pattern: the same sum, and the only form
    that stays affordable at m >= 32 (numpy evaluates the stacked einsum without
    intermediates, at O(r m^6))."""
    state.move_centre(n)
    t = state.T[n]
    if term_by_term:
        terms = state.heff_terms(n)

        def apply(x):
            return state.heff_apply(n, x, terms)
    else:
        stacked = state.heff_stacked(n)

        def apply(x):
            return state.heff_apply_stacked(x, stacked)

    e_cur = float(np.vdot(t, apply(t)) / np.vdot(t, t))
    theta, v, info = lanczos_lowest(apply, t, depth=depth, tol=tol)
    if theta <= e_cur + 1e-14 * abs(e_cur):
        state.set_tensor(n, v)
        return theta
    return e_cur


def ttn_sweep(state, depth=20, tol=1e-13, order=None, term_by_term=False):
    order = order or state.tree.post_order()
    e = None
    energies = []
    for n in order:
        e = local_step(state, n, depth, tol, term_by_term)
        energies.append(e)
    return e, energies


def attn_ground_state(state, terms, des, n_sweeps, s_ttn=1, us=None, depth=20, tol=1e-13,
                      de_max_iter=20, de_rel_dev=1e-12, log=None, term_by_term=False):
    """Run the schedule; returns (energies per sweep, disentanglers, local energies)."""
    us = [np.eye(4) for _ in des] if us is None else [u.copy() for u in us]
    out = []
    for s in range(n_sweeps):
        if s >= s_ttn and des:
            # isometric form is needed for the RDMs: the centre is wherever the
            # last sweep left it; RDMs are evaluated there.
            probs = build_problems(state, terms, des)
            us = [optimise_de(p, u, de_max_iter, de_rel_dev)[0] for p, u in zip(probs, us)]
        mapped = map_terms(terms, des, us)
        state.set_products(products_of(mapped))
        e, _ = ttn_sweep(state, depth, tol, term_by_term=term_by_term)
        out.append(e)
        if log:
            log(s, e)
    return out, us
