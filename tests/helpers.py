"""Shared helpers for the tests (no arithmetic of the method here)."""
from __future__ import annotations

import functools

import numpy as np

from oracle.group import Group
from workloads import cluster


def bits_for(two_s: int) -> int:
    b = 1
    while (1 << b) < two_s + 1:
        b += 1
    return b


def pack_labels(labels, n_sites: int, two_s: int) -> np.ndarray:
    """Re-encode base-(2s+1) labels (Eq. 2) as packed bit-field labels (site k in field k)."""
    d = two_s + 1
    bits = bits_for(two_s)
    out = np.zeros(len(labels), dtype=np.uint64)
    lab = np.array(labels, dtype=object)
    for k in range(n_sites):
        dig = np.array([int(v) % d for v in lab], dtype=np.uint64)
        out |= dig << np.uint64(bits * k)
        lab = np.array([int(v) // d for v in lab], dtype=object)
    return out


def unpack_label(p: int, n_sites: int, two_s: int) -> int:
    d = two_s + 1
    bits = bits_for(two_s)
    mask = (1 << bits) - 1
    n = 0
    for k in reversed(range(n_sites)):
        n = n * d + ((int(p) >> (bits * k)) & mask)
    return n


@functools.lru_cache(maxsize=None)
def oracle_group(name: str) -> Group:
    c = cluster(name)
    return Group(c.gens, c.bonds)


def masks_from_words(words: np.ndarray, G: int) -> np.ndarray:
    """Oracle stabilizer words (W x u64) -> [n, 2] u64 (128-bit masks)."""
    out = np.zeros((words.shape[0], 2), dtype=np.uint64)
    out[:, 0] = words[:, 0]
    if words.shape[1] > 1:
        out[:, 1] = words[:, 1]
    return out
