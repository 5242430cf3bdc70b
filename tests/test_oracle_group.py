"""Oracle pins: group closure and irreps (Section 3's verification: unitarity, orthogonality, completeness)."""
import numpy as np
import pytest

from oracle.group import Group, close_group
from workloads import cluster

# Known irrep dimensions of the point groups (character tables of I_h, O_h, T_d, D_5).
KNOWN = {
    "icosahedron": (120, [1, 1, 3, 3, 3, 3, 4, 4, 5, 5]),
    "dodecahedron": (120, [1, 1, 3, 3, 3, 3, 4, 4, 5, 5]),
    "icosidodecahedron": (120, [1, 1, 3, 3, 3, 3, 4, 4, 5, 5]),
    "cuboctahedron": (48, [1, 1, 1, 1, 2, 2, 3, 3, 3, 3]),
    "tetrahedron": (24, [1, 1, 2, 3, 3]),
    "ring:5": (10, [1, 1, 2, 2]),
    "dimer": (2, [1, 1]),
    "square:4x4": (128, None),
    "square:4x6": (96, None),
}


@pytest.mark.parametrize("name", sorted(KNOWN))
def test_irreps(name):
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    order, dims = KNOWN[name]
    assert g.order == order
    if dims is not None:
        assert [ir.dim for ir in g.irreps] == dims
    res = g.verify_irreps()
    assert res["sum_d2"] == order
    assert res["hom"] < 1e-12 and res["orth"] < 1e-12 and res["char"] < 1e-10 and res["row_orth"] < 1e-10
    assert all(ir.fs == 1 for ir in g.irreps)
    # identity first, trivial irrep first
    assert list(g.perms[0]) == list(range(c.n_sites))
    assert np.allclose(g.irreps[0].chars, 1.0)
    # characters are class functions with integer-valued d*chi/|C| central characters
    for ir in g.irreps:
        for cls in g.classes:
            assert np.allclose(ir.chars[cls], ir.chars[cls[0]], atol=1e-10)


def test_ih_sum_of_dims():
    """Section 2.3: sum_Gamma d_Gamma / sum_Gamma d_Gamma^2 = 32/120 for I_h."""
    g = Group(cluster("icosahedron").gens)
    assert sum(ir.dim for ir in g.irreps) == 32


def test_closure_rejects_non_permutation():
    with pytest.raises(ValueError):
        close_group([[0, 0, 1]])


def test_bond_invariance_check():
    c = cluster("icosahedron")
    bonds = np.array(c.bonds[:-1])
    with pytest.raises(ValueError):
        Group(c.gens, bonds)


def test_canonical_order_is_lexicographic():
    g = Group(cluster("cuboctahedron").gens)
    rows = [tuple(p) for p in g.perms.tolist()]
    assert rows == sorted(rows)
    assert len(set(rows)) == len(rows)
