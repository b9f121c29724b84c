"""Seeded random vectors: right-hand sides and finite-difference directions."""
import numpy as np


def uniform_rhs(n, nrhs=1, seed=1, low=-1.0, high=1.0):
    """n x nrhs FP64 entries uniform in [low, high] (a 1-D array when nrhs == 1)."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(low, high, size=(n, nrhs))
    return b[:, 0].copy() if nrhs == 1 else b


def unit_directions(shape, count, seed=7):
    """`count` seeded random directions of the given shape, each of unit 2-norm."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = rng.standard_normal(shape)
        out.append(d / np.linalg.norm(d))
    return out
