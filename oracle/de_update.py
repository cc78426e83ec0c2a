"""MERA-like disentangler update (Sec. 4.1, Eqs. energy, contracted, cost function).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Energy split (Eq. energy): with restriction (1), the energy is
E = sum_k sum_{p in P_k} E_k^p(u_k) + const, where P_k are the original terms
touching a site of disentangler k. For such a term on sites S_p, with
S'_p = S_p U {i, j} (at most three sites) and rho_p the TTN's reduced density
matrix on S'_p,
    E_k^p(u) = Tr[rho_p (u (x) 1)^T h_p (u (x) 1)].
Fixing the transposed factor at the current u_old makes the energy linear in
u, E = Tr(u Gamma_k) (Eq. contracted), with
    Gamma_k = sum_p Tr_extra[rho_p (u_old (x) 1)^T h~_p].
The minimiser over orthogonal u is u = -V W^T for Gamma_k = W sigma V^T, giving
Tr(u Gamma_k) = -sum sigma (Eq. cost function). The update is iterated
self-consistently; the environments (here the RDMs) are not recomputed.

Readings:
* The oracle builds Gamma_k from reduced density matrices of the TTN instead
  of the paper's left/right path environments (Sec. 4.2); both are the same
  contraction of the network around u_k, grouped differently.
* Shift: each term is shifted, h~_p = h_p - lambda_p 1 with lambda_p its
  spectral norm, so that h~_p <= 0 (standard MERA practice; the shift adds a
  u-independent constant to the true energy).
* A step is accepted only when the true E_k does not increase; iteration
  stops after ``max_iter`` = 20 steps or when the relative change is below
  ``rel_dev`` = 1e-12 (the paper names both parameters without values).

RDMs: rho[x, y] = <psi| (|x><y| (x) 1) |psi>, obtained as expectation values of
the 4^k rank-1 matrix-unit products, renormalised to the isometry centre with
the same link-by-link contraction as the effective operators.

Pins: RDMs equal those of the dense 16-site state; after an update
Tr(u Gamma) = -sum sigma; E_k(u) equals the dense energy difference.
"""
import numpy as np

from .disentangle import embed
from .ttn import TTNState


def partial_trace_keep(op, sites, keep):
    """Trace an operator on ``sites`` over every site not in ``keep`` (both ascending)."""
    k = len(sites)
    t = op.reshape([2] * (2 * k))
    drop = [a for a, s in enumerate(sites) if s not in keep]
    # trace pairs (a, a + k) from the highest axis down
    cur_k = k
    for a in sorted(drop, reverse=True):
        t = np.trace(t, axis1=a, axis2=a + cur_k)
        cur_k -= 1
    kk = len(keep)
    return t.reshape(2 ** kk, 2 ** kk)


def rdms(state, site_sets):
    """Reduced density matrices of the TTN on each ascending tuple of sites."""
    e = [np.zeros((2, 2)) for _ in range(4)]
    for a in range(4):
        e[a][a // 2, a % 2] = 1.0  # |x><y| with x = a // 2, y = a % 2
    prods = []
    index = []
    for w, sites in enumerate(site_sets):
        k = len(sites)
        for code in range(4 ** k):
            digs = [(code // 4 ** (k - 1 - b)) % 4 for b in range(k)]
            prods.append((tuple(sites), [e[d] for d in digs], w))
            index.append((w, digs))
    probe = TTNState(state.tree, state.T, state.centre, prods)
    n = probe.centre
    t = probe.T[n]
    ops = [probe.link_ops(n, s) for s in range(3)]
    out = [np.zeros((2 ** len(s), 2 ** len(s))) for s in site_sets]
    for q, (w, digs) in enumerate(index):
        y = t
        for s in range(3):
            o = ops[s].get(q)
            if o is not None:
                from .ttn import mode_product
                y = mode_product(y, o, s)
        val = float(np.vdot(t, y)) / float(np.vdot(t, t))
        xs = [d // 2 for d in digs]
        ys = [d % 2 for d in digs]
        xi = int("".join(map(str, xs)), 2)
        yi = int("".join(map(str, ys)), 2)
        out[w][xi, yi] = val
    return out


class DEProblem:
    """Everything the update of one disentangler needs: its terms and their RDMs."""

    def __init__(self, de, terms, rho):
        self.de = de
        self.terms = terms  # list of (S'_p, h_p embedded on S'_p, lambda_p)
        self.rho = rho      # list of RDMs on S'_p

    def energy(self, u):
        e = 0.0
        i, j = self.de
        for (sp, h, _), r in zip(self.terms, self.rho):
            U = embed(u, (i, j), sp)
            e += float(np.trace(r @ U.T @ h @ U))
        return e

    def gamma(self, u_old):
        i, j = self.de
        g = np.zeros((4, 4))
        for (sp, h, lam), r in zip(self.terms, self.rho):
            U = embed(u_old, (i, j), sp)
            ht = h - lam * np.eye(h.shape[0])
            g += partial_trace_keep(r @ U.T @ ht, sp, (i, j))
        return g


def build_problems(state, terms, des):
    """One DEProblem per disentangler (the RDMs of the current TTN)."""
    owner = {}
    for k, (i, j) in enumerate(des):
        owner[i] = owner[j] = k
    per = [[] for _ in des]
    for sites, op in terms:
        ks = {owner[x] for x in sites if x in owner}
        if not ks:
            continue
        k = ks.pop()
        i, j = des[k]
        sp = tuple(sorted(set(sites) | {i, j}))
        h = embed(op, tuple(sites), sp)
        lam = float(np.linalg.norm(op, 2))
        per[k].append((sp, h, lam))
    sets = []
    for k in range(len(des)):
        for sp, _, _ in per[k]:
            sets.append(sp)
    rho_all = rdms(state, sets) if sets else []
    out = []
    c = 0
    for k in range(len(des)):
        n = len(per[k])
        out.append(DEProblem(des[k], per[k], rho_all[c:c + n]))
        c += n
    return out


def optimise_de(problem, u0, max_iter=20, rel_dev=1e-12):
    """Self-consistent update u <- -V W^T (Sec. 4.1.1). Returns (u, E_k history)."""
    u = u0.copy()
    e = problem.energy(u)
    hist = [e]
    for _ in range(max_iter):
        g = problem.gamma(u)
        w, s, vt = np.linalg.svd(g)
        un = -(vt.T @ w.T)
        en = problem.energy(un)
        if en > e + 1e-14 * max(1.0, abs(e)):
            break
        done = abs(en - e) <= rel_dev * max(abs(e), 1e-300)
        u, e = un, en
        hist.append(e)
        if done:
            break
    return u, hist


# ------------------------------------------------ Riemannian gradient descent
# Sec. 4.1.2: both u and u^T vary; the cost is the true E_k(u) on the orthogonal
# group. Reading (the paper names the approach, not its parameters): Riemannian
# conjugate gradients in the embedded metric, Polak-Ribiere+ directions carried to
# the new point by projection, the QR retraction R_u(xi) = qf(u + xi) (positive
# diagonal of R), Armijo backtracking (c1 = 1e-4, halving) from a step of Frobenius
# norm 0.25 (doubled after an accepted step, at most 1), the same stopping rule as
# the MERA-like update (relative change below rel_dev, or max_iter steps).

def euclidean_gradient(problem, u):
    """dE_k/du = sum_p Tr_extra[2 h_p U rho_p], U = u (x) 1 on S'_p (h_p, rho_p symmetric)."""
    i, j = problem.de
    g = np.zeros((4, 4))
    for (sp, h, _), r in zip(problem.terms, problem.rho):
        U = embed(u, (i, j), sp)
        g += partial_trace_keep(2.0 * h @ U @ r, sp, (i, j))
    return g


def tangent(u, z):
    """Projection of z onto the tangent space of O(4) at u: u skew(u^T z)."""
    a = u.T @ z
    return u @ (0.5 * (a - a.T))


def retract(u, xi):
    q, r = np.linalg.qr(u + xi)
    return q * np.sign(np.diag(r))


def optimise_de_riemannian(problem, u0, max_iter=20, rel_dev=1e-12):
    """Riemannian conjugate-gradient minimisation of E_k over O(4). Returns (u, E_k history)."""
    u = u0.copy()
    e = problem.energy(u)
    hist = [e]
    g = tangent(u, euclidean_gradient(problem, u))
    d = -g
    step = 0.25
    for _ in range(max_iter):
        gd = float(np.sum(g * d))
        if not gd < 0.0:
            d, gd = -g, -float(np.sum(g * g))
        dn = float(np.linalg.norm(d))
        if dn == 0.0:
            break
        t = step / dn
        accepted = False
        for _ in range(40):
            un = retract(u, t * d)
            en = problem.energy(un)
            if en <= e + 1e-4 * t * gd:
                accepted = True
                break
            t *= 0.5
        if not accepted:
            break
        step = min(1.0, 2.0 * t * dn)
        gn = tangent(un, euclidean_gradient(problem, un))
        g_old = tangent(un, g)
        d_old = tangent(un, d)
        beta = max(0.0, float(np.sum(gn * (gn - g_old))) / max(float(np.sum(g * g)), 1e-300))
        done = abs(en - e) <= rel_dev * max(abs(e), 1e-300)
        u, e, g, d = un, en, gn, -gn + beta * d_old
        hist.append(e)
        if done:
            break
    return u, hist
