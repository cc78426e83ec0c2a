"""Learned disentangler initialiser, FP64 reference (not in the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper initialises every disentangler as the identity (Sec. 6). This
optional extra predicts a starting u_k from the TTN's two-site reduced density
matrix on the disentangler's sites:
    x  = rho_{ij} flattened row-major (16 reals),
    h1 = tanh(W1 x + b1)        (128),
    h2 = tanh(W2 h1 + b2)       (128),
    M  = W3 h2 + b3             (16, read row-major as 4 x 4),
    A  = (M - M^T) / 2          (antisymmetric generator),
    u  = expm(A)                (in SO(4)).
Loss per batch: mean over samples of ||u - u_target||_F^2. The backward pass
goes through the matrix exponential with its Frechet derivative: for real
matrices the gradient with respect to A is L(A^T, G_u) where L(A, E) is the
Frechet derivative of expm at A in direction E (library routine here).
Adam (Kingma and Ba 2015) with bias correction updates the weights.

Targets with det u_target = -1 cannot be reached by expm of a real
antisymmetric matrix; they are replaced by u_target diag(1, 1, 1, -1)
(reading; the disentangler update that follows starts from the prediction
and is judged by the true energy).

Pins: finite-difference gradients of the loss; expm(A) orthogonal to 1e-13.
"""
import numpy as np
from scipy.linalg import expm, expm_frechet

from inputs import normal

SIZES = (16, 128, 128, 16)


def init_params(seed):
    """Weights N(0, 1/fan_in), biases zero; stream 100 + layer."""
    p = {}
    for k in range(3):
        fi, fo = SIZES[k], SIZES[k + 1]
        p[f"W{k + 1}"] = normal(seed, 100 + k, fo * fi).reshape(fo, fi) / np.sqrt(fi)
        p[f"b{k + 1}"] = np.zeros(fo)
    return p


def canonical_target(u):
    if np.linalg.det(u) < 0:
        u = u @ np.diag([1.0, 1.0, 1.0, -1.0])
    return u


def forward(p, x):
    """x: [B, 16] -> (u [B, 4, 4], cache)."""
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    m = h2 @ p["W3"].T + p["b3"]
    mm = m.reshape(-1, 4, 4)
    A = 0.5 * (mm - np.transpose(mm, (0, 2, 1)))
    u = np.stack([expm(a) for a in A])
    return u, (x, h1, h2, A)


def loss_and_grad(p, x, ut):
    u, (x, h1, h2, A) = forward(p, x)
    B = x.shape[0]
    diff = u - ut
    loss = float(np.sum(diff * diff)) / B
    gu = 2.0 * diff / B
    gA = np.stack([expm_frechet(a.T, g, compute_expm=False) for a, g in zip(A, gu)])
    gm = 0.5 * (gA - np.transpose(gA, (0, 2, 1)))
    gm = gm.reshape(B, 16)
    g = {}
    g["W3"] = gm.T @ h2
    g["b3"] = gm.sum(0)
    gh2 = gm @ p["W3"]
    ga2 = gh2 * (1.0 - h2 * h2)
    g["W2"] = ga2.T @ h1
    g["b2"] = ga2.sum(0)
    gh1 = ga2 @ p["W2"]
    ga1 = gh1 * (1.0 - h1 * h1)
    g["W1"] = ga1.T @ x
    g["b1"] = ga1.sum(0)
    return loss, g


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for k in params:
            g = grads[k]
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * g
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * g * g
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            params[k] = params[k] - self.lr * mh / (np.sqrt(vh) + self.eps)
