"""Fixtures shared by the GPU parity tests: product group with the oracle's tabulated irreps."""
from __future__ import annotations

import functools

import numpy as np

from helpers import oracle_group
from workloads import cluster


def ftlm():
    from paper_2607_17429_gb300 import build

    build.build()
    from paper_2607_17429_gb300 import ftlm as F

    return F


@functools.lru_cache(maxsize=None)
def product_group(name: str):
    """Library group for ``name`` carrying the oracle's irrep matrices (Section 2.3: tabulated irreps)."""
    F = ftlm()
    c = cluster(name)
    og = oracle_group(name)
    g = F.ftlm_group_init(c.gens, c.bonds)
    F.ftlm_group_set_irreps(g, [ir.rho for ir in og.irreps])
    info = F.ftlm_group_info(g)
    assert np.abs(info["chars"] - og.char_table).max() < 1e-12
    return g


def torch_cuda():
    import torch

    assert torch.cuda.is_available()
    return torch
