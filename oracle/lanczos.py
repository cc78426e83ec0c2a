"""Lanczos local eigensolver (Sec. 4.4.2: "solving the local eigenproblem with
the Lanczos algorithm"; the method defers details to the DMRG literature).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Readings: Krylov space built from the current centre tensor, depth <= 20,
full reorthogonalisation (classical Gram-Schmidt applied twice), the
tridiagonal projection solved by a dense symmetric eigensolver (library step),
stop when the Ritz residual beta_k |y_k| < 1e-13 |theta| or on breakdown
(beta < 1e-300 or beta < 1e-14 * |alpha|-scale). Returns the lowest Ritz pair.

Pin: the lowest Ritz value of a full-depth run equals the dense lowest
eigenvalue of the same operator; every Ritz value is >= lambda_min.
"""
import numpy as np


def lanczos_lowest(apply, v0, depth=20, tol=1e-13):
    """Lowest Ritz pair of the symmetric operator ``apply`` from start vector v0.

    Returns (theta, vector (unit norm, same shape as v0), info dict)."""
    shape = v0.shape
    v = v0.reshape(-1) / np.linalg.norm(v0)
    basis = [v]
    alpha, beta = [], []
    theta, y = None, None
    for k in range(depth):
        w = apply(basis[k].reshape(shape)).reshape(-1)
        a = float(basis[k] @ w)
        alpha.append(a)
        w = w - a * basis[k]
        if k > 0:
            w = w - beta[k - 1] * basis[k - 1]
        vb = np.stack(basis)
        for _ in range(2):
            w = w - vb.T @ (vb @ w)
        b = float(np.linalg.norm(w))
        tmat = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        ev, evec = np.linalg.eigh(tmat)
        theta, y = float(ev[0]), evec[:, 0]
        scale = max(abs(theta), 1e-300)
        if b * abs(y[-1]) < tol * scale or b < 1e-14 * scale:
            break
        beta.append(b)
        basis.append(w / b)
    vb = np.stack(basis[: len(y)])
    x = y @ vb
    x /= np.linalg.norm(x)
    return theta, x.reshape(shape), {"iters": len(alpha), "alpha": alpha, "beta": beta}
