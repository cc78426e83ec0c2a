"""Isometrised binary TTN, effective operators and H_eff (Secs. 3.1, 3.3.2, 4.4.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Isometry (Sec. 3.1, Figs. unitary-tensor, iso): every tensor but the
  isometry centre satisfies T^T T = 1 when contracted over the two links that
  do not point towards the centre. Initial tensors are raw N(0,1) arrays
  (shared seeded input); each non-centre tensor is replaced by the Q factor of
  the QR decomposition of its (child0 child1) x parent matrix, with R's
  diagonal made non-negative; the centre (left top tensor) is normalised.
* Moving the centre (Fig. iso): QR of the tensor with the crossed link last;
  Q stays, R is multiplied into the neighbour on that link.
* Effective operators (Sec. 3.3.2, Fig. eff-op): computed separately for every
  TPO term -- here every rank-1 product of a mapped term -- by contracting the
  network around the tensor: an operator on link (n, s) is the product's
  one-site operators on the region behind that link, renormalised link by
  link with O_out = T^T (O_a (x) O_b) T over a tensor's two other links.
  Link operators are cached per (tensor, slot) and dropped when a tensor they
  depend on changes.
* H_eff x (Sec. 3.3.2 last paragraph, Sec. 4.4.2, Fig. eff-op-cost): every
  product's effective operators are contracted with the order-3 tensor one
  term after the other and the results are added; no term is summed with
  another before being applied.

Pins: isometry to 1e-12; for 16 sites the explicit embedding P (all tensors
but the centre) gives H_eff = P^T H' P and <T|H_eff|T> = <psi|H'|psi>.
"""
import numpy as np


def mode_product(t, a, slot):
    """(a x_slot t)[.., i, ..] = sum_j a[i, j] t[.., j, ..]."""
    return np.moveaxis(np.tensordot(a, t, axes=(1, slot)), 0, slot)


def qr_pos(mat):
    """Reduced QR with R's diagonal >= 0."""
    q, r = np.linalg.qr(mat)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s, r * s[:, None]


def renormalise(t, open_slot, ops):
    """O[t', t] = sum T[.., t', ..] (ops (x) ...) T[.., t, ..] over the two other slots.

    ``ops`` maps slot -> matrix (missing or None = identity)."""
    w = t
    for s, a in ops.items():
        if a is not None:
            w = mode_product(w, a, s)
    k = t.shape[open_slot]
    tm = np.moveaxis(t, open_slot, -1).reshape(-1, k)
    wm = np.moveaxis(w, open_slot, -1).reshape(-1, k)
    return tm.T @ wm


class TTNState:
    """Tensors of a binary TTN with an isometry centre and per-link operator caches."""

    def __init__(self, tree, tensors, centre, products=None):
        self.tree = tree
        self.T = [np.array(t, dtype=np.float64) for t in tensors]
        self.centre = centre
        self._far = {}
        self.set_products(products or [])

    # ------------------------------------------------------------ construction
    @classmethod
    def from_raw(cls, tree, raw, products=None):
        t0, _ = tree.top_nodes()
        ts = []
        for n in range(tree.n_nodes):
            a = np.array(raw[n], dtype=np.float64).reshape(tree.shape[n])
            if n == t0:
                ts.append(a / np.linalg.norm(a))
            else:
                d0, d1, d2 = a.shape
                q, _ = qr_pos(a.reshape(d0 * d1, d2))
                ts.append(q.reshape(d0, d1, d2))
        return cls(tree, ts, t0, products)

    def copy(self):
        s = TTNState(self.tree, [t.copy() for t in self.T], self.centre, self.products)
        return s

    def set_products(self, products):
        """Install the rank-1 products (sites, [ops], term) of the Hamiltonian in use."""
        self.products = list(products)
        self.site_prods = {}
        for q, (sites, ops, _) in enumerate(self.products):
            for s, o in zip(sites, ops):
                self.site_prods.setdefault(s, []).append((q, o))
        self.cache = {}

    # --------------------------------------------------------------- caching
    def far(self, n, slot):
        key = (n, slot)
        if key not in self._far:
            self._far[key] = self.tree.far_nodes(n, slot)
        return self._far[key]

    def set_tensor(self, n, t):
        self.T[n] = np.array(t, dtype=np.float64)
        dead = [k for k in self.cache if n in self.far(*k)]
        for k in dead:
            del self.cache[k]

    # ------------------------------------------------------------ isometries
    def isometry_error(self):
        """max over non-centre tensors of ||T^T T - 1|| towards the centre."""
        err = 0.0
        for n in range(self.tree.n_nodes):
            if n == self.centre:
                continue
            path = self.tree.path(n, self.centre)
            s = self.tree.slot_towards(n, path[1])
            t = np.moveaxis(self.T[n], s, -1)
            k = t.shape[-1]
            m = t.reshape(-1, k)
            err = max(err, float(np.abs(m.T @ m - np.eye(k)).max()))
        return err

    def move_centre(self, target):
        path = self.tree.path(self.centre, target)
        for a, b in zip(path[:-1], path[1:]):
            s = self.tree.slot_towards(a, b)
            back = self.tree.slot_towards(b, a)
            t = np.moveaxis(self.T[a], s, -1)
            shp = t.shape
            q, r = qr_pos(t.reshape(-1, shp[-1]))
            assert q.shape[1] == shp[-1], "link wider than its other side"
            self.set_tensor(a, np.moveaxis(q.reshape(shp), -1, s))
            self.set_tensor(b, mode_product(self.T[b], r, back))
            self.centre = b

    # --------------------------------------------------- effective operators
    def link_ops(self, n, slot):
        """{product q: renormalised operator on link (n, slot)} for products with
        at least one site behind that link (as seen from n)."""
        key = (n, slot)
        if key in self.cache:
            return self.cache[key]
        assert self.centre not in self.far(n, slot), "link not isometric towards n"
        kind, a, back = self.tree.nbr[n][slot]
        if kind == "site":
            out = {q: o for q, o in self.site_prods.get(a, [])}
        else:
            others = [s for s in range(3) if s != back]
            sub = {s: self.link_ops(a, s) for s in others}
            keys = sorted(set(sub[others[0]]) | set(sub[others[1]]))
            tc = self.T[a]
            out = {}
            for q in keys:
                out[q] = renormalise(tc, back, {s: sub[s].get(q) for s in others})
        self.cache[key] = out
        return out

    def heff_terms(self, n):
        """Per product: [op on slot 0, slot 1, slot 2] (None = identity)."""
        ops = [self.link_ops(n, s) for s in range(3)]
        out = []
        for q in range(len(self.products)):
            mats = [ops[s].get(q) for s in range(3)]
            if any(m is not None for m in mats):
                out.append(mats)
        return out

    def heff_apply(self, n, x, terms=None):
        """y = H_eff x, term by term (the definition)."""
        if terms is None:
            terms = self.heff_terms(n)
        y = np.zeros_like(x)
        for mats in terms:
            w = x
            for s in range(3):
                if mats[s] is not None:
                    w = mode_product(w, mats[s], s)
            y += w
        return y

    def heff_stacked(self, n):
        """The same term list grouped by which slots carry an operator, stacked."""
        groups = {}
        for mats in self.heff_terms(n):
            pat = tuple(m is not None for m in mats)
            groups.setdefault(pat, []).append([m for m in mats if m is not None])
        return {p: [np.stack([g[i] for g in gl]) for i in range(len(gl[0]))] for p, gl in groups.items()}

    def heff_apply_stacked(self, x, stacked):
        """y = sum over products of (ops) x, written as one einsum per slot pattern."""
        y = np.zeros_like(x)
        letters = "abc"
        inner = "ijk"
        for pat, mats in stacked.items():
            subs = []
            out = list(inner)
            for s in range(3):
                if pat[s]:
                    subs.append("r" + letters[s] + inner[s])
                    out[s] = letters[s]
            expr = ",".join(subs) + "," + inner + "->" + "".join(out)
            y += np.einsum(expr, *mats, x, optimize=True)
        return y

    def energy(self):
        """<T|H_eff|T>/<T|T> at the centre (= <psi|H'|psi> with the isometric form)."""
        n = self.centre
        t = self.T[n]
        return float(np.vdot(t, self.heff_apply(n, t)) / np.vdot(t, t))

    # ------------------------------------------------------------ dense (small N)
    def subtree_state(self, n):
        """Array [2^(sites of n), parent dim] of the subtree below node n."""
        tr = self.tree
        t = self.T[n]
        if tr.layer[n] == 1:
            return t.reshape(-1, t.shape[2])
        a = self.subtree_state(tr.nbr[n][0][1])
        b = self.subtree_state(tr.nbr[n][1][1])
        return np.einsum("ia,jb,abp->ijp", a, b, t).reshape(-1, t.shape[2])

    def dense(self):
        t0, t1 = self.tree.top_nodes()
        return (self.subtree_state(t0) @ self.subtree_state(t1).T).reshape(-1)

    def embedding(self, n):
        """P with psi = P vec(T_n): columns are dense states with T_n = unit tensors."""
        saved = self.T[n]
        cols = []
        for i in range(saved.size):
            e = np.zeros(saved.size)
            e[i] = 1.0
            self.T[n] = e.reshape(saved.shape)
            cols.append(self.dense())
        self.T[n] = saved
        return np.stack(cols, axis=1)


def heff_apply_ops(x, h_int=(None, None, None), pairs=None, triples=None):
    """Explicit-operator H_eff (the summed-link form of a node's term list).

    y = sum_l H_l x_l x + sum over pair kinds (p, q) and products r of
    (A_r on slot p) (B_r on slot q) x + sum over triples (O0, O1, O2) x.
    ``pairs`` maps (p, q) -> (A [R, m_p, m_p], B [R, m_q, m_q]); ``triples`` is
    (O0 [R, ..], O1, O2). Written term by term.
    """
    y = np.zeros_like(x)
    for s, h in enumerate(h_int):
        if h is not None:
            y += mode_product(x, h, s)
    for (p, q), (a, b) in (pairs or {}).items():
        for r in range(a.shape[0]):
            y += mode_product(mode_product(x, b[r], q), a[r], p)
    if triples is not None:
        o0, o1, o2 = triples
        for r in range(o0.shape[0]):
            y += mode_product(mode_product(mode_product(x, o2[r], 2), o1[r], 1), o0[r], 0)
    return y


def heff_sample_ops(x, idx, h_int=(None, None, None), pairs=None, triples=None):
    """Selected entries y[a, b, c] of the explicit-operator H_eff, one at a time.

    Each entry is an independent sum over the products (used for full-size
    sampled parity, where the whole product would take too long)."""
    out = np.zeros(len(idx))
    for e, (a, b, c) in enumerate(idx):
        v = 0.0
        if h_int[0] is not None:
            v += h_int[0][a] @ x[:, b, c]
        if h_int[1] is not None:
            v += h_int[1][b] @ x[a, :, c]
        if h_int[2] is not None:
            v += h_int[2][c] @ x[a, b, :]
        for (p, q), (A, B) in (pairs or {}).items():
            ia = (a, b, c)[p]
            iq = (a, b, c)[q]
            # slice of x with slots p, q free, the third fixed
            third = 3 - p - q
            xs = np.take(x, (a, b, c)[third], axis=third)  # 2-D [m_p, m_q]
            # sum_r A_r[ia, :] xs B_r[iq, :]^T
            v += float(np.einsum("ri,ij,rj->", A[:, ia, :], xs, B[:, iq, :]))
        if triples is not None:
            o0, o1, o2 = triples
            v += float(np.einsum("ri,rj,rk,ijk->", o0[:, a, :], o1[:, b, :], o2[:, c, :], x))
        out[e] = v
    return out
