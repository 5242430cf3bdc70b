"""Seeded random arrays used as H·v inputs in parity tests and the benchmark."""
from __future__ import annotations

import numpy as np


def rand_block_vectors(dim: int, B: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Return a [dim, B] array of i.i.d. standard normal entries (numpy PCG64, ``seed``).

    The layout matches the block-vector layout of the library: row (r, k) of the
    symmetry-adapted block, B right-hand sides contiguous per row.
    """
    rng = np.random.default_rng(seed)
    return rng.standard_normal((dim, B)).astype(dtype)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    z = z + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def label_keyed_values(keys, n_k: int, B: int, seed: int) -> np.ndarray:
    """Block-vector entries that depend only on (representative label, k, b, seed).

    keys: base-(2s+1) labels of representatives (the paper's Eq. 2 encoding).
    Returns [len(keys), n_k, B] values in [-1, 1).  Lets a block vector be built
    from any representative table and checked row by row without that table.
    """
    keys = np.asarray(keys, dtype=np.uint64).reshape(-1, 1, 1)
    k = np.arange(n_k, dtype=np.uint64).reshape(1, -1, 1)
    b = np.arange(B, dtype=np.uint64).reshape(1, 1, -1)
    with np.errstate(over="ignore"):
        z = keys * np.uint64(4096) + k * np.uint64(64) + b + np.uint64(seed) * np.uint64(0x632BE59BD9B4E019)
        h = _splitmix64(z)
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0
