"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This package holds no arithmetic of the method itself: it only builds cluster
geometries (sites, nearest-neighbour bonds, site-permutation generators of the
point or space group) and seeded random arrays.  Both the CUDA library and the
CPU oracle receive these as plain inputs.
"""
from .clusters import Cluster, cluster, CLUSTER_NAMES  # noqa: F401
from .seeded import label_keyed_values, rand_block_vectors  # noqa: F401
