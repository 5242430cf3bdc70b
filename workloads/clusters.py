"""Cluster geometries used as synthetic workloads.

Every cluster is built from coordinates: vertices of the polyhedron (or the
sites of a periodic lattice), nearest-neighbour bonds found by distance, and
the generators of the symmetry group as site permutations found by applying
the rotation/reflection to every vertex and matching the nearest vertex.  The
site permutation of a generator is stored as ``perm[k] = pi_g(k)``, the site
that site k is carried to (Section 2.3 of the paper: the digits of a label are
permuted by pi_g).

The bond counts of the polyhedra (30, 30, 60, 24) and their group orders
(I_h: 120, O_h: 48) are those of Table 1 and Section 3 of the paper.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PHI = (1.0 + math.sqrt(5.0)) / 2.0


@dataclasses.dataclass(frozen=True)
class Cluster:
    name: str
    n_sites: int
    bonds: np.ndarray  # int32 [n_bonds, 2], i < j, sorted
    gens: np.ndarray  # int32 [n_gens, n_sites], gens[g, k] = pi_g(k)
    coords: np.ndarray | None = None

    @property
    def n_bonds(self) -> int:
        return int(self.bonds.shape[0])


def _rot(axis, angle):
    u = np.asarray(axis, dtype=float)
    u = u / np.linalg.norm(u)
    ux = np.array([[0, -u[2], u[1]], [u[2], 0, -u[0]], [-u[1], u[0], 0]])
    return math.cos(angle) * np.eye(3) + math.sin(angle) * ux + (1 - math.cos(angle)) * np.outer(u, u)


def _perm_from_matrix(R, V):
    W = V @ R.T
    d = np.linalg.norm(W[:, None, :] - V[None, :, :], axis=2)
    p = np.argmin(d, axis=1)
    if not np.allclose(d[np.arange(len(V)), p], 0.0, atol=1e-9):
        raise ValueError("operation does not map the vertex set onto itself")
    if len(set(p.tolist())) != len(V):
        raise ValueError("operation is not a bijection of the vertices")
    return p.astype(np.int32)


def _nn_bonds(V):
    d = np.linalg.norm(V[:, None, :] - V[None, :, :], axis=2)
    dmin = np.min(d[d > 1e-9])
    ii, jj = np.nonzero(np.triu(np.isclose(d, dmin, rtol=1e-9, atol=1e-9), 1))
    b = np.stack([ii, jj], axis=1).astype(np.int32)
    return b[np.lexsort((b[:, 1], b[:, 0]))]


def _icosahedron_vertices():
    V = []
    for a in (1.0, -1.0):
        for b in (PHI, -PHI):
            V += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    return np.array(V)


def _dodecahedron_vertices():
    V = [(x, y, z) for x in (1.0, -1.0) for y in (1.0, -1.0) for z in (1.0, -1.0)]
    # Oriented as the dual of the icosahedron above (C5 axes through its vertices).
    for a in (PHI, -PHI):
        for b in (1.0 / PHI, -1.0 / PHI):
            V += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    return np.array(V)


def _icosidodecahedron_vertices():
    V = _icosahedron_vertices()
    E = _nn_bonds(V)
    return np.array([(V[i] + V[j]) / 2.0 for i, j in E])


def _cuboctahedron_vertices():
    V = []
    for a in (1.0, -1.0):
        for b in (1.0, -1.0):
            V += [(a, b, 0.0), (a, 0.0, b), (0.0, a, b)]
    return np.array(V)


def _ih_generators(V):
    c5 = _rot((0.0, 1.0, PHI), 2 * math.pi / 5)
    c3 = _rot((1.0, 1.0, 1.0), 2 * math.pi / 3)
    inv = -np.eye(3)
    return np.stack([_perm_from_matrix(M, V) for M in (c5, c3, inv)])


def _oh_generators(V):
    c4 = _rot((0.0, 0.0, 1.0), math.pi / 2)
    c3 = _rot((1.0, 1.0, 1.0), 2 * math.pi / 3)
    inv = -np.eye(3)
    return np.stack([_perm_from_matrix(M, V) for M in (c4, c3, inv)])


def _polyhedron(name, V, gens_fn):
    return Cluster(name=name, n_sites=len(V), bonds=_nn_bonds(V), gens=gens_fn(V), coords=V)


def _tetrahedron():
    V = np.array([(1.0, 1.0, 1.0), (1.0, -1.0, -1.0), (-1.0, 1.0, -1.0), (-1.0, -1.0, 1.0)])
    c3 = _rot((1.0, 1.0, 1.0), 2 * math.pi / 3)
    c2 = _rot((0.0, 0.0, 1.0), math.pi)
    mirror = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    gens = np.stack([_perm_from_matrix(M, V) for M in (c3, c2, mirror)])
    return Cluster("tetrahedron", 4, _nn_bonds(V), gens, V)


def _ring(n):
    """n-site ring with the dihedral group D_n (rotation by one site, reflection)."""
    if n < 3:
        raise ValueError("ring needs at least 3 sites")
    rot = np.array([(k + 1) % n for k in range(n)], dtype=np.int32)
    ref = np.array([(-k) % n for k in range(n)], dtype=np.int32)
    b = np.array(sorted(tuple(sorted((k, (k + 1) % n))) for k in range(n)), dtype=np.int32)
    return Cluster(f"ring:{n}", n, b, np.stack([rot, ref]))


def _chain(n):
    """n-site ring with its translations only (the cyclic group C_n: irreps of complex type for
    momenta k != 0, pi)."""
    if n < 3:
        raise ValueError("chain needs at least 3 sites")
    rot = np.array([(k + 1) % n for k in range(n)], dtype=np.int32)
    b = np.array(sorted(tuple(sorted((k, (k + 1) % n))) for k in range(n)), dtype=np.int32)
    return Cluster(f"chain:{n}", n, b, rot[None, :])


def _tetrahedron_rotations():
    """The tetrahedron with its rotation group T (order 12; one pair of complex-type irreps)."""
    V = np.array([(1.0, 1.0, 1.0), (1.0, -1.0, -1.0), (-1.0, 1.0, -1.0), (-1.0, -1.0, 1.0)])
    c3 = _rot((1.0, 1.0, 1.0), 2 * math.pi / 3)
    c2 = _rot((0.0, 0.0, 1.0), math.pi)
    gens = np.stack([_perm_from_matrix(M, V) for M in (c3, c2)])
    return Cluster("tetrahedron:t", 4, _nn_bonds(V), gens, V)


def _complete(p):
    """Complete graph on p sites (p prime) with the affine group x -> a x + b (mod p), a != 0:
    order p(p - 1), irreps of dimension 1 (some of complex type) and one of dimension p - 1."""
    if p < 3 or any(p % q == 0 for q in range(2, int(p ** 0.5) + 1)):
        raise ValueError("complete:p needs a prime p >= 3")
    root = next(a for a in range(2, p) if len({pow(a, e, p) for e in range(1, p)}) == p - 1)
    shift = np.array([(x + 1) % p for x in range(p)], dtype=np.int32)
    scale = np.array([(root * x) % p for x in range(p)], dtype=np.int32)
    b = np.array([(i, j) for i in range(p) for j in range(i + 1, p)], dtype=np.int32)
    return Cluster(f"complete:{p}", p, b, np.stack([shift, scale]))


def _petersen():
    """Petersen graph: sites are the 2-subsets of {0..4}, bonds join disjoint subsets; the group
    is S_5 acting on the subsets (order 120, irreps up to dimension 6)."""
    sub = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    index = {t: i for i, t in enumerate(sub)}

    def perm(f):
        return np.array([index[tuple(sorted((f[a], f[b])))] for a, b in sub], dtype=np.int32)

    gens = np.stack([perm([1, 2, 3, 4, 0]), perm([1, 0, 2, 3, 4])])
    bonds = np.array([(i, j) for i in range(10) for j in range(i + 1, 10) if not set(sub[i]) & set(sub[j])],
                     dtype=np.int32)
    return Cluster("petersen", 10, bonds, gens)


def _q8():
    """Cayley graph of the quaternion group Q_8 with connection set {+-i, +-j}; the group acts by
    left multiplication (order 8; one irrep of quaternionic type).  Site 2u + s is the unit
    u in (1, i, j, k) with sign (-1)^s."""
    # unit products: UNIT[u][v] = (w, sign) with u v = sign * w
    unit = [[(0, 1), (1, 1), (2, 1), (3, 1)],
            [(1, 1), (0, -1), (3, 1), (2, -1)],
            [(2, 1), (3, -1), (0, -1), (1, 1)],
            [(3, 1), (2, 1), (1, -1), (0, -1)]]

    def mul(x, y):
        (u, su), (v, sv) = divmod(x, 2), divmod(y, 2)
        w, sg = unit[u][v]
        neg = (su + sv + (sg < 0)) % 2
        return 2 * w + neg

    gens = np.stack([np.array([mul(g, x) for x in range(8)], dtype=np.int32) for g in (2, 4)])
    bonds = sorted({tuple(sorted((x, mul(x, c)))) for x in range(8) for c in (2, 4)})
    return Cluster("q8", 8, np.array(bonds, dtype=np.int32), gens)


def _dimer():
    return Cluster("dimer", 2, np.array([[0, 1]], dtype=np.int32), np.array([[1, 0]], dtype=np.int32))


def _square(lx, ly, pg):
    """lx x ly periodic square lattice; site k = x + lx*y.

    pg = "c4v" (needs lx == ly), "c2v" or "t" (translations only).
    """
    if lx < 3 or ly < 3:
        raise ValueError("square lattice needs lx, ly >= 3 (no doubled bonds)")

    def idx(x, y):
        return (x % lx) + lx * (y % ly)

    def perm(f):
        return np.array([idx(*f(k % lx, k // lx)) for k in range(lx * ly)], dtype=np.int32)

    gens = [perm(lambda x, y: (x + 1, y)), perm(lambda x, y: (x, y + 1))]
    if pg == "c4v":
        if lx != ly:
            raise ValueError("c4v needs a square torus")
        gens += [perm(lambda x, y: (-y, x)), perm(lambda x, y: (-x, y))]
    elif pg == "c2v":
        gens += [perm(lambda x, y: (-x, y)), perm(lambda x, y: (x, -y))]
    elif pg != "t":
        raise ValueError(f"unknown point group {pg!r}")
    bonds = set()
    for y in range(ly):
        for x in range(lx):
            for (u, v) in ((x + 1, y), (x, y + 1)):
                a, b = idx(x, y), idx(u, v)
                bonds.add((min(a, b), max(a, b)))
    b = np.array(sorted(bonds), dtype=np.int32)
    return Cluster(f"square:{lx}x{ly}:{pg}", lx * ly, b, np.stack(gens))


CLUSTER_NAMES = (
    "dimer", "tetrahedron", "tetrahedron:t", "icosahedron", "dodecahedron", "icosidodecahedron", "cuboctahedron",
    "ring:N", "chain:N", "square:LXxLY[:c4v|c2v|t]", "complete:P", "petersen", "q8",
)


def cluster(name: str) -> Cluster:
    """Build a cluster by name (see ``CLUSTER_NAMES``)."""
    if name == "dimer":
        return _dimer()
    if name == "tetrahedron":
        return _tetrahedron()
    if name == "tetrahedron:t":
        return _tetrahedron_rotations()
    if name == "petersen":
        return _petersen()
    if name == "q8":
        return _q8()
    if name.startswith("chain:"):
        return _chain(int(name.split(":")[1]))
    if name.startswith("complete:"):
        return _complete(int(name.split(":")[1]))
    if name == "icosahedron":
        return _polyhedron(name, _icosahedron_vertices(), _ih_generators)
    if name == "dodecahedron":
        return _polyhedron(name, _dodecahedron_vertices(), _ih_generators)
    if name == "icosidodecahedron":
        return _polyhedron(name, _icosidodecahedron_vertices(), _ih_generators)
    if name == "cuboctahedron":
        return _polyhedron(name, _cuboctahedron_vertices(), _oh_generators)
    if name.startswith("ring:"):
        return _ring(int(name.split(":")[1]))
    if name.startswith("square:"):
        parts = name.split(":")
        lx, ly = (int(v) for v in parts[1].split("x"))
        pg = parts[2] if len(parts) > 2 else ("c4v" if lx == ly else "c2v")
        return _square(lx, ly, pg)
    raise ValueError(f"unknown cluster {name!r}")
