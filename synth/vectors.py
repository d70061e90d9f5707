"""Seeded random vectors for operator-level parity tests."""
import numpy as np


def random_node_vectors(dim, n, count, seed):
    """count random node arrays of (n+1)^dim values (x fastest), zero on the boundary."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((count,) + (n + 1,) * dim)
    inner = (slice(None),) + (slice(1, n),) * dim
    out = np.zeros_like(v)
    out[inner] = v[inner]
    return out.reshape(count, -1)


def random_element_field(dim, n, count, seed, spread=1.0):
    """count positive per-element fields exp(spread * N(0,1)), n^dim values each."""
    rng = np.random.default_rng(seed)
    return np.exp(spread * rng.standard_normal((count, n ** dim)))
