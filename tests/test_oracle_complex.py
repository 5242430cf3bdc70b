"""Oracle pins for irreps of complex and quaternionic type, and for irrep dimensions above 5.

Section 3 keeps real arithmetic for irreps of real Frobenius-Schur type.  The oracle (and the
library) take every other irrep in its real form: a complex pair Gamma, conj(Gamma) as one real
representation of dimension 2 d_Gamma, a quaternionic Gamma as one of dimension 2 d_Gamma.  The
single-partner-row block of a real form holds every level of the complex block kappa times
(kappa = <chi_R, chi_R> = 2 or 4), so it enters Eqs. 5, 6 and 14 with weight dim / kappa.

Pins (none uses the block machinery to check itself):

* the real-form irrep lists of textbook groups: C_n, the rotation group T of the tetrahedron,
  the affine groups AGL(1, p) (one irrep of dimension p - 1), S_5 on the Petersen graph
  (dimensions 1, 1, 4, 4, 5, 5, 6), the quaternion group Q_8 (one quaternionic irrep);
* the dense projector check (Section 4.1) on their blocks: the explicit Eq. 12 vectors are
  orthonormal and Psi^T H Psi equals the pull-form H·v block;
* levels of a real-form block come in kappa-fold multiplets;
* the weighted union of all block spectra is the full sector spectrum (full ED), which pins
  the weight; a planted weight of dim instead of dim / kappa fails it;
* the complete graph K_p: H = (J/2)(S_tot^2 - p s(s+1)), levels and multiplicities in closed form;
* exact-mode thermodynamics (Eqs. 5-7) against full ED for clusters with complex irreps.
"""
import math

import numpy as np
import pytest

from oracle.basis import BlockBasis, SectorBasis
from oracle.dense import projected_basis, sector_hamiltonian
from oracle.group import Group
from oracle.lanczos import thermo
from oracle.sector import block_dims, sector_dim
from workloads import cluster

# (cluster, expected [(dim, indicator)] in canonical order)
IRREPS = {
    "chain:5": [(1, 1), (2, 0), (2, 0)],
    "chain:6": [(1, 1), (1, 1), (2, 0), (2, 0)],
    "chain:8": [(1, 1), (1, 1), (2, 0), (2, 0), (2, 0)],
    "tetrahedron:t": [(1, 1), (2, 0), (3, 1)],
    "complete:5": [(1, 1), (1, 1), (2, 0), (4, 1)],
    "complete:7": [(1, 1), (1, 1), (2, 0), (2, 0), (6, 1)],
    "complete:11": [(1, 1), (1, 1), (2, 0), (2, 0), (2, 0), (2, 0), (10, 1)],
    "petersen": [(1, 1), (1, 1), (4, 1), (4, 1), (5, 1), (5, 1), (6, 1)],
    "q8": [(1, 1), (1, 1), (1, 1), (1, 1), (4, -1)],
    "square:4x4:t": [(1, 1)] * 4 + [(2, 0)] * 6,
}


@pytest.mark.parametrize("name", sorted(IRREPS))
def test_real_form_irrep_lists(name):
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    assert [(ir.dim, ir.fs) for ir in g.irreps] == IRREPS[name]
    res = g.verify_irreps()
    assert res["hom"] < 1e-10 and res["orth"] < 1e-10 and res["char"] < 1e-10 and res["row_orth"] < 1e-10
    assert res["sum_d2"] == g.order
    for ir in g.irreps:
        assert ir.kappa * ir.weight == ir.dim
        # complex pair: chi_R = 2 Re chi has |chi_R(g)| <= dim with the identity alone at dim
        assert abs(ir.chars[0] - ir.dim) < 1e-12


DENSE = [("chain:5", 1, 1), ("chain:6", 2, 0), ("chain:8", 1, 0), ("tetrahedron:t", 3, 0), ("q8", 1, 0),
         ("q8", 2, 2), ("complete:5", 2, 0), ("complete:7", 1, 1), ("complete:11", 1, 5), ("petersen", 1, 0),
         ("petersen", 2, 4), ("square:4x4:t", 1, 8)]


def _blocks_and_sector(name, two_s, two_M):
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    sec = SectorBasis(g, two_s, two_M)
    labels, H = sector_hamiltonian(c.n_sites, two_s, two_M, c.bonds)
    blocks = [(ir, BlockBasis(sec, i).with_hamiltonian(c.bonds)) for i, ir in enumerate(g.irreps)]
    return c, g, labels, H, blocks


@pytest.mark.parametrize("name,two_s,two_M", DENSE)
def test_dense_check_multiplets_and_weighted_union(name, two_s, two_M):
    c, g, labels, H, blocks = _blocks_and_sector(name, two_s, two_M)
    ev = []
    for ir, blk in blocks:
        if blk.dim == 0:
            continue
        Psi = projected_basis(blk, labels)
        assert np.abs(Psi.T @ Psi - np.eye(blk.dim)).max() < 1e-12
        Hb = blk.dense()
        assert np.abs(Psi.T @ H @ Psi - Hb).max() < 1e-11
        e = np.linalg.eigvalsh(Hb)
        if ir.kappa > 1:  # kappa-fold multiplets
            assert blk.dim % ir.kappa == 0
            grp = e.reshape(-1, ir.kappa)
            assert np.abs(grp - grp[:, :1]).max() < 1e-9
        ev.extend(list(e) * ir.weight)
    ref = np.linalg.eigvalsh(H)
    assert len(ev) == len(ref)
    assert np.abs(np.sort(ev) - ref).max() < 1e-10


def test_planted_weight_fails_the_union():
    """Weight dim (the real-type rule) on a complex-type block over-counts its levels."""
    c, g, labels, H, blocks = _blocks_and_sector("chain:6", 2, 0)
    ev = []
    for ir, blk in blocks:
        if blk.dim:
            ev.extend(list(np.linalg.eigvalsh(blk.dense())) * ir.dim)
    assert len(ev) != len(H)


@pytest.mark.parametrize("p,two_s", [(5, 2), (7, 1), (11, 1), (5, 3)])
def test_complete_graph_closed_form(p, two_s):
    """K_p: every level is (J/2)(S(S+1) - p s(s+1)); over all M >= 0 blocks the weighted level
    counts equal (number of spin-S multiplets) x (2S+1), from the sector dimensions alone."""
    c = cluster(f"complete:{p}")
    g = Group(c.gens, c.bonds)
    s = two_s / 2
    counts = {}
    for two_M in range(p * two_s % 2, p * two_s + 1, 2):
        sec = SectorBasis(g, two_s, two_M)
        mult = 2 if two_M > 0 else 1
        for i, ir in enumerate(g.irreps):
            blk = BlockBasis(sec, i).with_hamiltonian(c.bonds)
            if blk.dim == 0:
                continue
            for e in np.linalg.eigvalsh(blk.dense()):
                S2 = 2 * e / 1.0 + p * s * (s + 1)  # S(S+1)
                S = (-1 + math.sqrt(1 + 4 * S2)) / 2
                Sr = round(2 * S) / 2
                assert abs(S - Sr) < 1e-9
                counts[Sr] = counts.get(Sr, 0) + mult * ir.weight
    ref = {}
    for two_S in range(p * two_s % 2, p * two_s + 1, 2):
        n_mult = sector_dim(p, two_s, two_S) - sector_dim(p, two_s, two_S + 2)
        if n_mult:
            ref[two_S / 2] = n_mult * (two_S + 1)
    assert counts == ref


@pytest.mark.parametrize("name,two_s", [("chain:6", 1), ("q8", 1), ("complete:5", 2), ("tetrahedron:t", 3)])
def test_thermo_exact_mode_with_weights(name, two_s):
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    N = c.n_sites
    blocks = []
    for two_M in range(N * two_s % 2, N * two_s + 1, 2):
        sec = SectorBasis(g, two_s, two_M)
        dims = block_dims(g, two_s, two_M)
        for i, ir in enumerate(g.irreps):
            blk = BlockBasis(sec, i).with_hamiltonian(c.bonds)
            assert blk.dim == dims[i]  # character formula with chi_R
            if blk.dim == 0:
                continue
            e = np.linalg.eigvalsh(blk.dense())
            blocks.append(dict(two_M=two_M, d_gamma=ir.weight, dim=blk.dim, R=blk.dim,
                               alpha=[np.array([v]) for v in e], beta=[np.array([0.0]) for _ in e]))
    T = np.geomspace(0.05, 50, 30)
    lnZ, E, C, chi, _ = thermo(blocks, T, g=2.0)
    Es, Msq = [], []
    for two_M in range(-N * two_s, N * two_s + 1, 2):
        _, H = sector_hamiltonian(N, two_s, two_M, c.bonds)
        e = np.linalg.eigvalsh(H)
        Es += list(e)
        Msq += [(two_M / 2) ** 2] * len(e)
    Es, Msq = np.array(Es), np.array(Msq)
    for t, temp in enumerate(T):
        b = 1 / temp
        w = np.exp(-b * (Es - Es.min()))
        Z = w.sum()
        Em = (w * Es).sum() / Z
        assert np.isclose(lnZ[t], np.log(Z) - b * Es.min(), rtol=1e-10)
        assert np.isclose(E[t], Em, rtol=1e-9, atol=1e-10)
        assert np.isclose(C[t], b * b * (w * (Es - Em) ** 2).sum() / Z, rtol=1e-8, atol=1e-10)
        assert np.isclose(chi[t], 4.0 * b * (w * Msq).sum() / Z, rtol=1e-9, atol=1e-12)
