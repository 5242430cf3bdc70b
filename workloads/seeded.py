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
