"""Counter-based SplitMix64 deviates (no method arithmetic lives here)."""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    """SplitMix64 output function applied elementwise to uint64 values."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed, stream):
    with np.errstate(over="ignore"):
        s = np.uint64(seed) * GOLDEN
        return mix64(s ^ mix64(np.uint64(stream) + np.uint64(1)))


def _bits(seed, stream, n, offset=0):
    k = _key(seed, stream)
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(k + i * GOLDEN)


def uniform(seed, stream, n):
    """n uniforms in [0, 1) from stream (seed, stream)."""
    b = _bits(seed, stream, n)
    return (b >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed, stream, n):
    """n standard normal deviates from stream (seed, stream), Box-Muller on pairs."""
    n2 = (n + 1) // 2
    u = uniform(seed, stream, 2 * n2).reshape(n2, 2)
    u1 = 1.0 - u[:, 0]  # (0, 1]
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u[:, 1]
    z = np.empty((n2, 2))
    z[:, 0] = r * np.cos(t)
    z[:, 1] = r * np.sin(t)
    return z.reshape(-1)[:n].copy()


def raw_tree_tensors(shapes, seed):
    """Raw N(0,1) tensors, one per tree node; node ``k`` draws stream ``k``.

    ``shapes`` is a list of 3-tuples (child0, child1, parent). Returns a list of
    float64 C-contiguous arrays of those shapes.
    """
    out = []
    for k, shp in enumerate(shapes):
        n = int(np.prod(shp))
        out.append(normal(seed, k, n).reshape(shp))
    return out


def random_vector(shape, seed, stream=1 << 20):
    """A random N(0,1) node-shaped vector (e.g. a Lanczos start or test input)."""
    n = int(np.prod(shape))
    return normal(seed, stream, n).reshape(shape)


def random_operators(count, dim, seed, stream, symmetric=True, scale=None):
    """``count`` random real dim x dim link operators, symmetric by default.

    Entries are N(0,1) scaled by 1/sqrt(dim) (so that the operator norm is O(1));
    symmetric operators are (G + G^T)/2 of that.
    """
    if scale is None:
        scale = 1.0 / np.sqrt(dim)
    g = normal(seed, stream, count * dim * dim).reshape(count, dim, dim) * scale
    if symmetric:
        g = 0.5 * (g + np.transpose(g, (0, 2, 1)))
    return np.ascontiguousarray(g)
