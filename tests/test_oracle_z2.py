"""Oracle pins for the spin-flip extension G x Z_2 at M = 0 (Section 2.2).

The global flip F: m_k -> -m_k (digits a_k -> 2s - a_k) commutes with H and with every
site permutation; irreps of G x Z_2 are Gamma+ and Gamma-.  Pins:

* dense projector check (Section 4.1) on Gamma+- blocks: the explicit Eq. 12 vectors of the
  extended group, Psi^T H Psi, equal the oracle's pull-form H·v block;
* those vectors are eigenvectors of F with eigenvalue +1 (Gamma+) or -1 (Gamma-);
* spec(Gamma+) u spec(Gamma-) = spec(Gamma) block by block (the split only refines);
* block dimensions: the character formula over G x Z_2 (flip-fixed states counted in
  closed form) equals the enumeration, and dim Gamma+ + dim Gamma- = dim Gamma;
* a planted mistake (Gamma- with the sign of Gamma+) fails the flip check.
"""
import copy

import numpy as np
import pytest

from oracle.basis import BlockBasis, SectorBasis, hv_rows_by_label
from oracle.dense import projected_basis, sector_hamiltonian
from oracle.group import Group, SpinFlipExtended
from oracle.sector import block_dims
from workloads import cluster

CASES = [("icosahedron", 1), ("tetrahedron", 2), ("tetrahedron", 3), ("cuboctahedron", 1), ("ring:6", 2),
         ("chain:6", 2), ("q8", 1), ("complete:5", 2)]  # the last three with real forms of complex/quaternionic irreps


def _flip_matrix(labels, n_sites, two_s):
    d = two_s + 1
    pos = {n: i for i, n in enumerate(labels)}
    Fm = np.zeros((len(labels), len(labels)))
    for i, n in enumerate(labels):
        m, dig = n, []
        for _ in range(n_sites):
            dig.append(m % d)
            m //= d
        f = 0
        for v in reversed(dig):
            f = f * d + (d - 1 - v)
        Fm[pos[f], i] = 1.0
    return Fm


@pytest.mark.parametrize("name,two_s", CASES)
def test_z2_dense_check_flip_parity_and_spectra(name, two_s):
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    gx = SpinFlipExtended(g)
    labels, H = sector_hamiltonian(c.n_sites, two_s, 0, c.bonds)
    Fm = _flip_matrix(labels, c.n_sites, two_s)
    assert np.abs(Fm @ H - H @ Fm).max() < 1e-12  # F commutes with H
    sec = SectorBasis(g, two_s, 0)
    secx = SectorBasis(gx, two_s, 0)
    assert secx.n_reps <= sec.n_reps
    for i, ir in enumerate(g.irreps):
        if ir.rho is None:
            continue
        parent = BlockBasis(sec, i).with_hamiltonian(c.bonds)
        ev = []
        for sgn, k in ((1, 2 * i), (-1, 2 * i + 1)):
            blk = BlockBasis(secx, k).with_hamiltonian(c.bonds)
            if blk.dim == 0:
                continue
            Psi = projected_basis(blk, labels)
            assert np.abs(Psi.T @ Psi - np.eye(blk.dim)).max() < 1e-12
            assert np.abs(Fm @ Psi - sgn * Psi).max() < 1e-12
            Hb = blk.dense()
            assert np.abs(Psi.T @ H @ Psi - Hb).max() < 1e-11
            ev.extend(np.linalg.eigvalsh(Hb))
        assert len(ev) == parent.dim
        if parent.dim:
            assert np.abs(np.sort(ev) - np.linalg.eigvalsh(parent.dense())).max() < 1e-10


@pytest.mark.parametrize("name,two_s", CASES + [("icosahedron", 3), ("dodecahedron", 1), ("dodecahedron", 3)])
def test_z2_block_dims_character_formula(name, two_s):
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    gx = SpinFlipExtended(g)
    dims = block_dims(g, two_s, 0)
    dimsx = block_dims(gx, two_s, 0)
    for i in range(len(g.irreps)):
        assert dimsx[2 * i] + dimsx[2 * i + 1] == dims[i]
    if name != "dodecahedron":  # enumeration is cheap only for the small clusters
        secx = SectorBasis(gx, two_s, 0)
        for k, ir in enumerate(gx.irreps):
            if ir.rho is not None:
                assert BlockBasis(secx, k).dim == dimsx[k]


def test_z2_label_keyed_rows_match_block_hv():
    c = cluster("icosahedron")
    gx = SpinFlipExtended(Group(c.gens, c.bonds))
    secx = SectorBasis(gx, 3, 0)
    rng = np.random.default_rng(4)
    for k in (0, 3, 9, 17):
        blk = BlockBasis(secx, k).with_hamiltonian(c.bonds)
        x = rng.standard_normal(blk.dim)
        y = blk.hv(x)
        sel = rng.choice(secx.n_reps, 40, replace=False)
        rows = hv_rows_by_label(gx, k, c.bonds, 1.0, 3, secx.reps[sel].tolist(),
                                lambda lab, n: x[blk.off[np.searchsorted(secx.reps, lab)]:][:n, None])
        for i, r in zip(sel, rows):
            if r is None:
                assert blk.n[i] == 0
                continue
            assert np.abs(r[:, 0] - y[blk.off[i]:blk.off[i + 1]]).max() < 1e-12


def test_z2_flip_check_catches_wrong_sign():
    c = cluster("icosahedron")
    g = Group(c.gens, c.bonds)
    gx = SpinFlipExtended(g)
    bad = copy.copy(gx)
    bad.irreps = list(gx.irreps)
    ir = gx.irreps[2 * 5 + 1]  # a Gamma- irrep given the rho of its Gamma+
    bad.irreps[2 * 5 + 1] = copy.copy(ir)
    bad.irreps[2 * 5 + 1].rho = gx.irreps[2 * 5].rho
    labels, H = sector_hamiltonian(c.n_sites, 1, 0, c.bonds)
    Fm = _flip_matrix(labels, c.n_sites, 1)
    secx = SectorBasis(bad, 1, 0)
    try:
        blk = BlockBasis(secx, 2 * 5 + 1).with_hamiltonian(c.bonds)
    except ArithmeticError:
        return  # the character count and the projector rank disagree: caught
    Psi = projected_basis(blk, labels)
    assert blk.dim == 0 or np.abs(Fm @ Psi + Psi).max() > 1e-3


def test_z2_split_of_table2():
    """Table 2 lists the s=3/2 dodecahedron's M = 0 blocks with the Gamma+- sub-blocks added back
    (Section 4.3): the character formula over G x Z_2 splits every entry into two parts."""
    import os

    c = cluster("dodecahedron")
    g = Group(c.gens, c.bonds)
    dimsx = block_dims(SpinFlipExtended(g), 3, 0)
    sums = sorted(dimsx[2 * i] + dimsx[2 * i + 1] for i in range(len(g.irreps)))
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_dodecahedron_s32_M0.txt")
    table = sorted(int(ln.split()[3]) for ln in open(path) if ln.strip() and not ln.startswith("#"))
    assert sums == table
    assert all(dimsx[k] > 0 for k in range(len(dimsx)))
