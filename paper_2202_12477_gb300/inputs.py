"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

Holds no arithmetic of the method: only numpy's PCG64 generator turned into
vectors of the sizes the operator takes. Mesh perturbations and right-hand
sides are not made here; both sides derive them from the counter-based
SplitMix64 generator defined in the C header.
"""
from __future__ import annotations

import numpy as np


def random_vector(n: int, seed: int, kind: str = "uniform") -> np.ndarray:
    """Length-n FP64 vector: 'uniform' in [-1, 1), 'normal' N(0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "uniform":
        return rng.uniform(-1.0, 1.0, size=n)
    if kind == "normal":
        return rng.standard_normal(size=n)
    raise ValueError(kind)


def sample_indices(n: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct indices in [0, n), sorted, always including 0 and n-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = min(count, n)
    idx = set(rng.choice(n, size=max(count - 2, 0), replace=False).tolist()) if n > 2 else set()
    idx.update({0, n - 1})
    return np.array(sorted(idx), dtype=np.int64)
