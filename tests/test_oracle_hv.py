"""Oracle pins for H·v: dense projector check (Section 4.1), full ED, SU(2) multiplets.

The dense check compares the oracle's pull-form H·v block with Psi^T H Psi, where
Psi holds the explicit symmetry-adapted vectors of Eq. 12 and H is Eq. 1 built
entry by entry.  The planted-mistake tests show that a transposed rho, a dropped
stabilizer ratio or a wrong connecting element g_e make this check fail.
"""
import copy

import numpy as np
import pytest

from oracle.basis import BlockBasis, SectorBasis
from oracle.dense import full_hamiltonian, projected_basis, sector_hamiltonian
from oracle.group import Group
from workloads import cluster

CASES = [("tetrahedron", 1, 0), ("tetrahedron", 3, 2), ("ring:5", 1, 1), ("ring:6", 3, 0),
         ("icosahedron", 1, 0), ("icosahedron", 1, 4), ("cuboctahedron", 1, 0), ("cuboctahedron", 2, 18),
         ("icosahedron", 3, 30), ("square:3x3:c4v", 1, 1)]


def _dense_check(g, c, two_s, two_M, mutate=None):
    sec = SectorBasis(g, two_s, two_M)
    labels, H = sector_hamiltonian(c.n_sites, two_s, two_M, c.bonds)
    worst = 0.0
    for ir in range(len(g.irreps)):
        blk = BlockBasis(sec, ir).with_hamiltonian(c.bonds)
        if blk.dim == 0:
            continue
        Psi = projected_basis(blk, labels)
        assert np.abs(Psi.T @ Psi - np.eye(blk.dim)).max() < 1e-12
        if mutate is not None:
            blk = mutate(blk)
        Hb = blk.dense()
        worst = max(worst, np.abs(Psi.T @ H @ Psi - Hb).max())
    return worst


@pytest.mark.parametrize("name,two_s,two_M", CASES)
def test_dense_projector_check(name, two_s, two_M):
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    assert _dense_check(g, c, two_s, two_M) < 1e-11


def _transpose_rho(blk):
    b = copy.copy(blk)
    b.rho = np.ascontiguousarray(np.transpose(blk.rho, (0, 2, 1)))
    return b


def _drop_ratio(blk):
    b = copy.copy(blk)
    b.sqrtS = np.ones_like(blk.sqrtS)
    return b


@pytest.mark.parametrize("mutate", [_transpose_rho, _drop_ratio])
def test_dense_check_catches_planted_mistakes(mutate):
    c = cluster("icosahedron")
    g = Group(c.gens, c.bonds)
    assert _dense_check(g, c, 1, 0, mutate) > 1e-3


def test_dense_check_catches_wrong_connecting_element():
    c = cluster("icosahedron")
    g = Group(c.gens, c.bonds)
    g2 = copy.copy(g)
    g2.inv = np.arange(g.order)  # uses g* instead of g_e = g*^{-1}
    sec = SectorBasis(g, 1, 0)
    labels, H = sector_hamiltonian(12, 1, 0, c.bonds)
    worst = 0.0
    for ir in range(len(g.irreps)):
        blk = BlockBasis(sec, ir).with_hamiltonian(c.bonds)
        Psi = projected_basis(blk, labels)
        sec2 = copy.copy(sec)
        sec2.group = g2
        blk2 = copy.copy(blk)
        blk2.sector = sec2
        worst = max(worst, np.abs(Psi.T @ H @ Psi - blk2.dense()).max())
    assert worst > 1e-3


def _all_block_spectra(name, two_s):
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    N = c.n_sites
    evs = []
    spec = {}
    for two_M in range(N * two_s % 2, N * two_s + 1, 2):
        sec = SectorBasis(g, two_s, two_M)
        mult = 2 if two_M > 0 else 1
        for ir in range(len(g.irreps)):
            blk = BlockBasis(sec, ir).with_hamiltonian(c.bonds)
            if blk.dim == 0:
                spec[(two_M, ir)] = np.zeros(0)
                continue
            Hb = blk.dense()
            assert np.abs(Hb - Hb.T).max() < 1e-12
            e = np.linalg.eigvalsh(Hb)
            spec[(two_M, ir)] = e
            evs.extend(list(e) * (mult * g.irreps[ir].weight))
    return c, g, np.sort(np.array(evs)), spec


def test_full_ed_icosahedron():
    """Union of all block spectra (times d_Gamma * mult_M) = spectrum of the 4096 x 4096 H."""
    c, g, evs, _ = _all_block_spectra("icosahedron", 1)
    H = full_hamiltonian(12, 1, c.bonds)
    ref = np.linalg.eigvalsh(H)
    assert len(evs) == 4096
    assert np.abs(evs - ref).max() < 1e-10


def test_full_ed_tetrahedron_spin2():
    c, g, evs, _ = _all_block_spectra("tetrahedron", 4)
    H = full_hamiltonian(4, 4, c.bonds)
    assert np.abs(evs - np.linalg.eigvalsh(H)).max() < 1e-10


@pytest.mark.parametrize("name,two_s", [("icosahedron", 1), ("cuboctahedron", 1), ("tetrahedron", 3)])
def test_su2_multiplets(name, two_s):
    """SU(2): every level of sector M+1 appears in sector M, same irrep; E_min(M) non-decreasing."""
    c, g, _, spec = _all_block_spectra(name, two_s)
    N = c.n_sites
    Ms = list(range(N * two_s % 2, N * two_s + 1, 2))
    for ir in range(len(g.irreps)):
        for m_lo, m_hi in zip(Ms[:-1], Ms[1:]):
            lo, hi = spec[(m_lo, ir)], spec[(m_hi, ir)]
            for e in hi:
                assert np.min(np.abs(lo - e)) < 1e-9
    emin = [min((spec[(m, ir)].min() for ir in range(len(g.irreps)) if len(spec[(m, ir)])), default=np.inf)
            for m in Ms]
    assert all(a <= b + 1e-10 for a, b in zip(emin[:-1], emin[1:]))


def test_dimer_spectrum_closed_form():
    """Two spins s: E(S) = (J/2)[S(S+1) - 2 s(s+1)], degeneracy 2S+1."""
    for two_s in (1, 2, 3, 5):
        s = two_s / 2
        _, _, evs, _ = _all_block_spectra("dimer", two_s)
        ref = []
        for twoS in range(0, 2 * two_s + 1, 2):
            S = twoS / 2
            ref += [0.5 * (S * (S + 1) - 2 * s * (s + 1))] * int(2 * S + 1)
        assert np.allclose(evs, np.sort(ref), atol=1e-12)


@pytest.mark.parametrize("name,two_s,two_M", CASES)
def test_hv_rows_by_label_matches_dense_checked_block_hv(name, two_s, two_M):
    """The table-free, label-keyed oracle rows (Eqs. 15-16 from each label alone) equal the rows of the
    dense-checked BlockBasis.hv on the same label-keyed input, for every irrep of every CASES sector."""
    from oracle.basis import hv_rows_by_label
    from workloads import label_keyed_values

    c = cluster(name)
    g = Group(c.gens, c.bonds)
    sec = SectorBasis(g, two_s, two_M)
    B = 3
    checked = 0
    for ir in range(len(g.irreps)):
        if g.irreps[ir].rho is None:
            continue
        blk = BlockBasis(sec, ir).with_hamiltonian(c.bonds)
        if blk.dim == 0:
            continue
        vals = label_keyed_values(sec.reps, max(1, int(blk.n.max())), B, 17 + ir)
        X = np.concatenate([vals[i, :blk.n[i]] for i in range(sec.n_reps)])
        Y = blk.hv(X)
        rows = hv_rows_by_label(g, ir, c.bonds, 1.0, two_s, sec.reps,
                                lambda lab, n, s=17 + ir: label_keyed_values([lab], n, B, s)[0])
        scale = np.abs(Y).max() + 1e-300
        for i, yr in enumerate(rows):
            if blk.n[i] == 0:
                assert yr is None
                continue
            assert yr.shape == (blk.n[i], B)
            assert np.abs(yr - Y[blk.off[i]:blk.off[i + 1]]).max() <= 1e-13 * scale
            checked += 1
    assert checked > 0
