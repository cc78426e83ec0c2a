"""Lattices, site order and the two benchmark Hamiltonians (Sec. 6).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Site order: the lattice is mapped to a line along a Hilbert curve before the
  tree is built (Sec. 6, "Hilbert curve mapping pattern"). We use the classic
  ``d2xy`` construction; site index == curve index.
* Transverse-field Ising model (Eq. qising). The paper prints it with the
  coupling on sigma_x and the field on sigma_z; we use the equivalent form
  H = -sum_<ij> Z_i Z_j - h sum_i X_i (a global Hadamard maps one to the
  other, so the spectrum is the same).
* Triangular-lattice Heisenberg model (Eq. xxz): the square lattice plus one
  diagonal, bonds (+1,0), (0,+1), (+1,+1), open boundaries, with spin-1/2
  operators S = sigma/2. Each bond contributes three separate terms
  Sx Sx, Sy Sy, Sz Sz (Sec. 6.2.2 counts them as separate TPO terms).
  Sy Sy is real: Y (x) Y = -(iY) (x) (iY) with iY = [[0,1],[-1,0]].
* Local terms acting on the same site are summed into one term (Sec. 3.3).

A term is (sites, op): ``sites`` is an ascending tuple of site indices and
``op`` a real 2^k x 2^k matrix whose row/column index lists the sites'
spins with the first (smallest) site most significant.

Pins: curve bijectivity and adjacency; TFIM exact energies from the oracle's
own sparse eigensolver versus a free-fermion closed form on a chain.
"""
import numpy as np

X = np.array([[0.0, 1.0], [1.0, 0.0]])
Z = np.array([[1.0, 0.0], [0.0, -1.0]])
IY = np.array([[0.0, 1.0], [-1.0, 0.0]])  # i * sigma_y, real
I2 = np.eye(2)


def hilbert_d2xy(n, d):
    """Curve index d -> (x, y) on an n x n grid (n a power of two)."""
    x = y = 0
    s = 1
    t = d
    while s < n:
        rx = 1 & (t // 2)
        ry = 1 & (t ^ rx)
        if ry == 0:
            if rx == 1:
                x = s - 1 - x
                y = s - 1 - y
            x, y = y, x
        x += s * rx
        y += s * ry
        t //= 4
        s *= 2
    return x, y


class Lattice:
    """Sites with coordinates, in curve order, plus a list of bonds (site pairs)."""

    def __init__(self, coords, bonds, name):
        self.coords = list(coords)
        self.n = len(self.coords)
        self.bonds = sorted((min(a, b), max(a, b)) for a, b in bonds)
        self.name = name


def square_lattice(L, triangular=False):
    """L x L open-boundary lattice in Hilbert order; triangular adds (+1,+1) bonds."""
    assert L >= 2 and (L & (L - 1)) == 0
    coords = [hilbert_d2xy(L, d) for d in range(L * L)]
    index = {c: i for i, c in enumerate(coords)}
    steps = [(1, 0), (0, 1)] + ([(1, 1)] if triangular else [])
    bonds = []
    for (x, y), i in index.items():
        for dx, dy in steps:
            nb = (x + dx, y + dy)
            if nb in index:
                bonds.append((i, index[nb]))
    return Lattice(coords, bonds, ("tri" if triangular else "square") + f"{L}x{L}")


def chain(n):
    """Open chain of n sites in natural order (used only for closed-form pins)."""
    return Lattice([(i, 0) for i in range(n)], [(i, i + 1) for i in range(n - 1)], f"chain{n}")


def sum_local_terms(terms):
    """Merge all one-site terms on the same site into one (Sec. 3.3)."""
    local = {}
    out = []
    for sites, op in terms:
        if len(sites) == 1:
            s = sites[0]
            local[s] = local.get(s, 0.0) + op
        else:
            out.append((sites, op))
    for s in sorted(local):
        out.append(((s,), local[s]))
    return out


def tfim_terms(lat, h):
    """H = -sum_<ij> Z_i Z_j - h sum_i X_i (Eq. qising with the coupling on Z, J = 1; same spectrum)."""
    terms = [((i, j), -np.kron(Z, Z)) for i, j in lat.bonds]
    terms += [((s,), -h * X) for s in range(lat.n)]
    return sum_local_terms(terms)


def heisenberg_terms(lat, J=1.0):
    """H = J sum_<ij> (Sx Sx + Sy Sy + Sz Sz), S = sigma/2 (Eq. xxz with spin-1/2 units)."""
    terms = []
    for i, j in lat.bonds:
        terms.append(((i, j), 0.25 * J * np.kron(X, X)))
        terms.append(((i, j), -0.25 * J * np.kron(IY, IY)))
        terms.append(((i, j), 0.25 * J * np.kron(Z, Z)))
    return terms


# ---------------------------------------------------------------- dense states

def apply_op(psi, n, sites, op):
    """Apply a k-site operator to a 2^n state vector (axis s = site s, site 0 most significant)."""
    k = len(sites)
    t = psi.reshape([2] * n)
    t = np.moveaxis(t, list(sites), list(range(k)))
    shp = t.shape
    t = (op @ t.reshape(2 ** k, -1)).reshape(shp)
    t = np.moveaxis(t, list(range(k)), list(sites))
    return t.reshape(-1)


def apply_terms(psi, n, terms):
    out = np.zeros_like(psi)
    for sites, op in terms:
        out += apply_op(psi, n, sites, op)
    return out


def energy_dense(psi, n, terms):
    return float(psi @ apply_terms(psi, n, terms)) / float(psi @ psi)


def ground_energy_ed(n, terms, tol=1e-12):
    """Lowest eigenvalue of sum(terms) on 2^n states (Sec. 4 exact reference).

    Uses scipy's implicitly restarted Lanczos on a matrix-free operator (a
    library eigensolver serving as one step).
    """
    from scipy.sparse.linalg import LinearOperator, eigsh

    dim = 2 ** n
    op = LinearOperator((dim, dim), matvec=lambda v: apply_terms(np.asarray(v).reshape(-1), n, terms),
                        dtype=np.float64)
    v0 = np.ones(dim) / np.sqrt(dim)
    w = eigsh(op, k=1, which="SA", tol=tol, v0=v0, return_eigenvectors=False)
    return float(w[0])


def tfim_chain_exact(n, h):
    """Closed-form OBC TFIM chain ground energy (free fermions, Pfeuty 1970).

    After the Jordan-Wigner transformation, H = -sum Z_i Z_{i+1} - h sum X_i is
    quadratic in Majorana operators; the field couples the two Majoranas of a
    site with weight h and each bond couples neighbouring sites with weight 1.
    The single-particle energies Lambda_k are the singular values of the
    bidiagonal n x n matrix M (diagonal h, super-diagonal 1) and
    E0 = -sum_k Lambda_k.
    """
    M = np.diag(np.full(n, float(h))) + np.diag(np.ones(n - 1), 1)
    s = np.linalg.svd(M, compute_uv=False)
    return -float(np.sum(s))
