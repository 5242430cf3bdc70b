"""Oracle pins: sector and block dimensions against the paper's tables and exact identities."""
import os

import numpy as np
import pytest

from oracle.basis import BlockBasis, SectorBasis
from oracle.group import Group
from oracle.sector import block_dims, sector_dim
from workloads import cluster

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_table1_sector_dims():
    for _, N, two_s, dfull, d0 in _rows("table1_sector_dims.txt"):
        N, two_s = int(N), int(two_s)
        assert (two_s + 1) ** N == int(dfull)
        assert sector_dim(N, two_s, 0) == int(d0)


def test_table2_block_dims():
    c = cluster("dodecahedron")
    g = Group(c.gens, c.bonds)
    dims = block_dims(g, 3, 0)
    inv = g.element(c.gens[2])  # the inversion generator
    got = sorted((ir.dim, int(np.sign(ir.chars[inv])), D) for ir, D in zip(g.irreps, dims))
    want = sorted((int(d), int(p), int(D)) for _, d, p, D in _rows("table2_dodecahedron_s32_M0.txt"))
    assert got == want
    assert sum(ir.dim * D for ir, D in zip(g.irreps, dims)) == sector_dim(20, 3, 0)


@pytest.mark.parametrize("name,two_s", [("icosahedron", 1), ("cuboctahedron", 2), ("tetrahedron", 3),
                                        ("ring:5", 3), ("icosidodecahedron", 1), ("square:4x4", 1)])
def test_completeness_over_sectors(name, two_s):
    """sum_M sum_Gamma d_Gamma D_{M,Gamma} = (2s+1)^N over every M."""
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    N = c.n_sites
    tot = 0
    for two_M in range(-N * two_s, N * two_s + 1, 2):
        tot += sum(ir.dim * D for ir, D in zip(g.irreps, block_dims(g, two_s, two_M)))
    assert tot == (two_s + 1) ** N


@pytest.mark.parametrize("name,two_s,two_M", [("icosahedron", 1, 0), ("icosahedron", 3, 2), ("cuboctahedron", 2, 0),
                                              ("tetrahedron", 3, 2), ("ring:6", 1, 0), ("square:4x4", 1, 0)])
def test_enumeration_matches_counting(name, two_s, two_M):
    """Brute-force orbits: rep count = Burnside count, sum n_Gamma(r) = character formula (Eq. 13)."""
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    sec = SectorBasis(g, two_s, two_M)
    from oracle.sector import fixed_count
    burnside = sum(fixed_count(p, two_s, two_M) for p in g.perms)
    assert burnside % g.order == 0
    assert sec.n_reps == burnside // g.order
    assert np.all(np.diff(sec.reps.astype(np.int64)) > 0)
    # every stabilizer is a subgroup: orbit length |G|/|Stab| sums to the sector dimension
    lengths = [g.order // len(sec.stab_elems[t]) for t in sec.stab_index]
    assert sum(lengths) == sector_dim(c.n_sites, two_s, two_M)
    dims = block_dims(g, two_s, two_M)
    for ir in range(len(g.irreps)):
        assert BlockBasis(sec, ir).dim == dims[ir]
