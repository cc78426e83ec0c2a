"""Binary tree geometry of the TTN (Sec. 3.1, Fig. attn).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Reading of "log2(N) - 1 layers": layer l = 1 .. nL (nL = log2 N - 1) holds
N / 2^l tensors; a layer-l tensor covers 2^l consecutive sites (in curve
order); layer 1 tensors carry the physical links; the top layer has two
tensors joined by one "top link". Every tensor is rank 3 with slots
(0 = left child, 1 = right child, 2 = parent). The link above a layer-l tensor
has dimension min(d^(2^l), m); the top link min(d^(N/2), m); physical links d.

Node ids: layer 1 first (left to right), then layer 2, ... , the two top
tensors last. ``node_id(l, j)`` gives the id of tensor j of layer l.

Pins: the link-dimension rule reproduces the shapes listed for the 4x4, m = 8
case; every (node, slot) triple of regions partitions the sites.
"""


def _cap_dim(d, exp2, m):
    """min(d^(2^exp2), m) without overflow."""
    if exp2 >= 7:
        return m
    return min(d ** (2 ** exp2), m)


class Tree:
    def __init__(self, n_sites, m, d=2):
        assert n_sites >= 4 and (n_sites & (n_sites - 1)) == 0
        self.n_sites = n_sites
        self.m = m
        self.d = d
        self.nL = n_sites.bit_length() - 2  # log2(N) - 1
        self.layer = []
        self.index = []
        self._id = {}
        for l in range(1, self.nL + 1):
            for j in range(n_sites >> l):
                self._id[(l, j)] = len(self.layer)
                self.layer.append(l)
                self.index.append(j)
        self.n_nodes = len(self.layer)
        # neighbour of (node, slot): ("site", s) or ("node", id, slot_on_that_node)
        self.nbr = []
        self.shape = []
        for n in range(self.n_nodes):
            l, j = self.layer[n], self.index[n]
            if l == 1:
                ch = [("site", 2 * j, None), ("site", 2 * j + 1, None)]
                cdim = d
            else:
                ch = [("node", self._id[(l - 1, 2 * j)], 2), ("node", self._id[(l - 1, 2 * j + 1)], 2)]
                cdim = _cap_dim(d, l - 1, m)
            if l < self.nL:
                par = ("node", self._id[(l + 1, j // 2)], j % 2)
                pdim = _cap_dim(d, l, m)
            else:
                par = ("node", self._id[(l, 1 - j)], 2)
                pdim = _cap_dim(d, self.nL, m)
            self.nbr.append([ch[0], ch[1], par])
            self.shape.append((cdim, cdim, pdim))

    def node_id(self, l, j):
        return self._id[(l, j)]

    def sites_of(self, n):
        """Sites covered by the subtree of node n (a consecutive range)."""
        l, j = self.layer[n], self.index[n]
        return range(j << l, (j + 1) << l)

    def region(self, n, slot):
        """Set of sites behind link ``slot`` of node n, as seen from n."""
        kind, a, _ = self.nbr[n][slot]
        if kind == "site":
            return {a}
        if slot < 2:
            return set(self.sites_of(a))
        inside = set(self.sites_of(n))
        return set(range(self.n_sites)) - inside

    def top_nodes(self):
        return self.node_id(self.nL, 0), self.node_id(self.nL, 1)

    def path(self, a, b):
        """Node ids from a to b along the unique tree path (inclusive)."""
        if a == b:
            return [a]

        def up(n):
            chain = [n]
            while self.layer[chain[-1]] < self.nL:
                chain.append(self.nbr[chain[-1]][2][1])
            return chain

        ua, ub = up(a), up(b)
        if ua[-1] != ub[-1]:
            return ua + ub[::-1]
        sb = set(ub)
        i = 0
        while ua[i] not in sb:
            i += 1
        lca = ua[i]
        return ua[: i + 1] + ub[: ub.index(lca)][::-1]

    def slot_towards(self, n, nb):
        """Slot of node n whose link leads to the adjacent node nb."""
        for s in range(3):
            kind, a, _ = self.nbr[n][s]
            if kind == "node" and a == nb:
                return s
        raise ValueError("not adjacent")

    def far_nodes(self, n, slot):
        """Nodes on the far side of link (n, slot)."""
        kind, a, back = self.nbr[n][slot]
        if kind == "site":
            return set()
        out = set()
        stack = [(a, back)]
        while stack:
            c, bslot = stack.pop()
            out.add(c)
            for s in range(3):
                if s == bslot:
                    continue
                k2, a2, b2 = self.nbr[c][s]
                if k2 == "node":
                    stack.append((a2, b2))
        return out

    def post_order(self):
        """Sweep order: post-order of the left top subtree, then of the right one."""
        order = []

        def visit(n):
            if self.layer[n] > 1:
                visit(self.nbr[n][0][1])
                visit(self.nbr[n][1][1])
            order.append(n)

        t0, t1 = self.top_nodes()
        visit(t0)
        visit(t1)
        return order

    def lca_layer(self, i, j):
        """Layer of the lowest tensor whose subtree holds sites i and j; nL+1 if
        they lie in different top halves (the top link is then the highest
        link between them)."""
        for l in range(1, self.nL + 1):
            if (i >> l) == (j >> l):
                return l
        return self.nL + 1
