"""Disentangler placement and the mapping H -> H' (Secs. 3.2, 4.3, 6.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Placement (Sec. 6.1.2): loop over the candidate positions, highest supported
link first, and accept a pair of sites when it lies fully on a Hamiltonian
interaction term and violates neither restriction of Sec. 6.1.1:
  (1) no Hamiltonian term may touch more than one disentangler;
  (2) a disentangler must not support untruncated links.
Readings: candidates are the two-site interaction terms (bonds); the
"supported" link of a pair (i, j) is the highest link on the tree path between
them, i.e. a child link of their lowest common tensor (the top link when they
lie in different top halves); it is truncated when m < d^(2^(l-1)) for a
lowest common tensor of layer l. Ties at equal layer are broken by the
ascending site pair. Placement stops at the requested count; the number
actually placed is reported by the caller.

Mapping (Sec. 4.3, Algorithm 1, Fig. DE-MPO-contr): for every term and every
disentangler whose sites intersect the term's sites, the term becomes
u^T (h (x) 1) u on the union of the sites (case (a): the disentangler lies
fully on the term; case (b): an identity is inserted on the extra site).
Reading of the conjugation order: the state is |psi_aTTN> = D |psi_TTN>
(Eq. attn), so <psi_aTTN|H|psi_aTTN> = <psi_TTN|D^T H D|psi_TTN>; we keep that
and call the mapped operator H' = D^T H D (the paper's D H D^dagger with D
renamed). All quantities are real (both models are real symmetric), so the
dagger is a transpose. A disentangler u on sites (i, j), i < j, is a 4 x 4
matrix with site i's spin most significant.

Products: each mapped term on k <= 3 sites is split exactly into rank-1
tensor products of one-site operators by successive SVDs (site by site, in
ascending site order), dropping singular values below 1e-14 of the largest.
A two-site term therefore has at most d^2 = 4 products (the bond-dimension
bound of Sec. 4.3).

Pins: restrictions (1)/(2) hold on every placement; for 4 x 4 the dense
D^T H D equals the sum of the mapped terms on random states; every product
list reassembles its term.
"""
import numpy as np


def embed(op, sites, target):
    """Extend an operator on ``sites`` to the ascending ``target`` superset (identity elsewhere)."""
    k, kt = len(sites), len(target)
    if tuple(sites) == tuple(target):
        return op
    extra = [s for s in target if s not in sites]
    full = np.kron(op, np.eye(2 ** len(extra)))
    order = list(sites) + extra  # current axis order of full's row (and column) index
    perm = [order.index(s) for s in target]
    t = full.reshape([2] * (2 * kt))
    t = np.transpose(t, perm + [p + kt for p in perm])
    return t.reshape(2 ** kt, 2 ** kt)


def place_disentanglers(tree, terms, max_de):
    """Greedy placement of Sec. 6.1.2; returns the accepted (i, j) pairs, i < j."""
    nL, m, d = tree.nL, tree.m, tree.d
    bonds = sorted({tuple(s) for s, _ in terms if len(s) == 2})
    site_terms = {}
    for s, _ in terms:
        for x in s:
            site_terms.setdefault(x, []).append(tuple(s))

    def truncated(l):
        e = 2 ** (l - 1)
        return e >= 7 or m < d ** e

    cands = sorted(bonds, key=lambda p: (-tree.lca_layer(*p), p[0], p[1]))
    owner = {}  # site -> index of its disentangler
    placed = []
    for i, j in cands:
        if len(placed) >= max_de:
            break
        if i in owner or j in owner:
            continue
        if not truncated(tree.lca_layer(i, j)):
            continue
        ok = True
        for s in site_terms.get(i, []) + site_terms.get(j, []):
            if any(x in owner for x in s):
                ok = False
                break
        if not ok:
            continue
        owner[i] = owner[j] = len(placed)
        placed.append((i, j))
    return placed


def check_restrictions(tree, terms, des):
    """True when no term touches two disentanglers and none sits on untruncated links."""
    owner = {}
    for k, (i, j) in enumerate(des):
        if i in owner or j in owner:
            return False
        owner[i] = owner[j] = k
        l = tree.lca_layer(i, j)
        e = 2 ** (l - 1)
        if not (e >= 7 or tree.m < tree.d ** e):
            return False
    for s, _ in terms:
        if len({owner[x] for x in s if x in owner}) > 1:
            return False
    return True


def map_terms(terms, des, us):
    """H' = D^T H D term by term (Algorithm 1). ``us[k]`` is the 4x4 disentangler on ``des[k]``."""
    owner = {}
    for k, (i, j) in enumerate(des):
        owner[i] = owner[j] = k
    out = []
    for sites, op in terms:
        ks = {owner[x] for x in sites if x in owner}
        assert len(ks) <= 1, "restriction (1) violated"
        if not ks:
            out.append((tuple(sites), op))
            continue
        k = ks.pop()
        i, j = des[k]
        target = tuple(sorted(set(sites) | {i, j}))
        h = embed(op, sites, target)
        u = embed(us[k], (i, j), target)
        out.append((target, u.T @ h @ u))
    return out


def split_products(sites, op, rel_cut=1e-14):
    """Exact rank-1 split of a term into products of one-site operators.

    Returns a list of lists of 2x2 matrices (one per site, ascending)."""
    k = len(sites)
    if k == 1:
        return [[op.copy()]]
    # tensor with index order (s1, s1', s2, s2', ...)
    t = op.reshape([2] * (2 * k))
    perm = []
    for a in range(k):
        perm += [a, a + k]
    t = np.transpose(t, perm).reshape([4] * k)

    def rec(tt):
        # tt: array whose first index is the current site's (s, s') pair
        if tt.ndim == 1:
            return [[tt.reshape(2, 2)]]
        mat = tt.reshape(4, -1)
        u, s, vt = np.linalg.svd(mat, full_matrices=False)
        if s[0] == 0.0:
            return []
        keep = s > rel_cut * s[0]
        res = []
        for a in np.nonzero(keep)[0]:
            head = (u[:, a] * s[a]).reshape(2, 2)
            rest = vt[a].reshape(tt.shape[1:])
            for tail in rec(rest):
                res.append([head] + tail)
        return res

    return rec(t)


def products_of(terms, rel_cut=1e-14):
    """Flatten mapped terms into rank-1 products: list of (sites, [ops]) with a term index."""
    prods = []
    for t, (sites, op) in enumerate(terms):
        for ops in split_products(sites, op, rel_cut):
            prods.append((tuple(sites), ops, t))
    return prods


def reassemble(sites, ops_list):
    """Sum over products of kron(ops) (used by pins)."""
    acc = 0.0
    for ops in ops_list:
        o = ops[0]
        for x in ops[1:]:
            o = np.kron(o, x)
        acc = acc + o
    return acc
