"""Oracle pins for the FTLM driver: Philox KAT, Lanczos sum rule, exact thermal sums, high-T limit."""
import os

import numpy as np
import pytest

from oracle.basis import BlockBasis, SectorBasis
from oracle.dense import sector_hamiltonian
from oracle.group import Group
from oracle.lanczos import lanczos, philox4x32_10, ritz, start_vectors, thermo
from workloads import cluster

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = philox4x32_10(*v[:4], v[4], v[5])
        assert [int(o) for o in out] == v[6:]


def test_start_vectors_statistics():
    x = start_vectors(200000, 2, seed=7, block_id=3)
    assert np.allclose(np.sum(x * x, axis=0), 1.0, atol=1e-14)
    z = x[:, 0] * np.sqrt(200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.02
    assert abs(np.mean(z ** 4) - 3) < 0.1  # Gaussian kurtosis
    assert abs(np.corrcoef(x[:, 0], x[:, 1])[0, 1]) < 0.01
    r = start_vectors(1000, 1, seed=7, block_id=3, rng="rademacher")
    assert np.allclose(np.abs(r), 1 / np.sqrt(1000))
    # different blocks/chains/seeds give different streams
    assert not np.allclose(start_vectors(64, 1, 7, 3), start_vectors(64, 1, 7, 4))
    assert not np.allclose(start_vectors(64, 1, 7, 3), start_vectors(64, 1, 8, 3))


def _block(name, two_s, two_M, ir):
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    return BlockBasis(SectorBasis(g, two_s, two_M), ir).with_hamiltonian(c.bonds)


def test_lanczos_sum_rule_and_exhaustion():
    blk = _block("icosahedron", 1, 0, 9)  # H_u-like 5-dim irrep block, dim < 60
    v0 = start_vectors(blk.dim, 1, 0, 0)[:, 0]
    a, b = lanczos(blk.hv, v0, 60)
    assert len(a) <= blk.dim
    th, w = ritz(a, b)
    assert abs(w.sum() - 1) < 1e-12
    H = blk.dense()
    ev, U = np.linalg.eigh(H)
    # Ritz values carrying weight lie on the spectrum once the Krylov space is exhausted
    for t, wk in zip(th, w):
        if wk > 1e-8:
            assert np.min(np.abs(ev - t)) < 1e-8
    # and the quadrature is exact for exp(-H): <v0|e^{-H}|v0> = sum_k w_k e^{-theta_k}
    exact = np.sum((U.T @ v0) ** 2 * np.exp(-ev))
    assert np.isclose(np.sum(w * np.exp(-th)), exact, rtol=1e-10)


def test_lanczos_tridiagonal_reproduces_moments():
    """<v0|H^p|v0> = sum_k w_k theta_k^p for p < 2m (Krylov exactness)."""
    blk = _block("icosahedron", 1, 2, 0)
    H = blk.dense()
    v0 = start_vectors(blk.dim, 1, 1, 5)[:, 0]
    a, b = lanczos(blk.hv, v0, 4)
    th, w = ritz(a, b)
    for p in range(8):
        assert np.isclose(v0 @ np.linalg.matrix_power(H, p) @ v0, np.sum(w * th ** p), rtol=1e-9, atol=1e-9)


def _exact_blocks(name, two_s):
    """Every (M, Gamma) block as 'chains' that are its eigenvectors: FTLM in exact mode."""
    c = cluster(name)
    g = Group(c.gens, c.bonds)
    N = c.n_sites
    blocks = []
    for two_M in range(N * two_s % 2, N * two_s + 1, 2):
        sec = SectorBasis(g, two_s, two_M)
        for ir in range(len(g.irreps)):
            blk = BlockBasis(sec, ir).with_hamiltonian(c.bonds)
            if blk.dim == 0:
                continue
            e = np.linalg.eigvalsh(blk.dense())
            blocks.append(dict(two_M=two_M, d_gamma=g.irreps[ir].weight, dim=blk.dim, R=blk.dim,
                               alpha=[np.array([v]) for v in e], beta=[np.array([0.0]) for _ in e]))
    return c, blocks


def _ed_thermo(name, two_s, T, g=1.0):
    c = cluster(name)
    N = c.n_sites
    E, Msq = [], []
    for two_M in range(-N * two_s, N * two_s + 1, 2):
        _, H = sector_hamiltonian(N, two_s, two_M, c.bonds)
        e = np.linalg.eigvalsh(H)
        E += list(e)
        Msq += [(two_M / 2) ** 2] * len(e)
    E, Msq = np.array(E), np.array(Msq)
    out = []
    for t in T:
        b = 1 / t
        w = np.exp(-b * (E - E.min()))
        Z = w.sum()
        Em = (w * E).sum() / Z
        out.append((np.log(Z) - b * E.min(), Em, b * b * ((w * (E - Em) ** 2).sum() / Z), g * g * b * (w * Msq).sum() / Z))
    return np.array(out).T


@pytest.mark.parametrize("name,two_s", [("icosahedron", 1), ("tetrahedron", 3), ("dimer", 3), ("ring:5", 1)])
def test_thermo_exact_mode_matches_full_ed(name, two_s):
    T = np.geomspace(0.02, 100, 40)
    _, blocks = _exact_blocks(name, two_s)
    lnZ, E, C, chi, E0 = thermo(blocks, T, g=2.0)
    ref = _ed_thermo(name, two_s, T, g=2.0)
    assert np.allclose(lnZ, ref[0], rtol=1e-10)
    assert np.allclose(E, ref[1], rtol=1e-9, atol=1e-10)
    assert np.allclose(C, ref[2], rtol=1e-8, atol=1e-10)
    assert np.allclose(chi, ref[3], rtol=1e-9, atol=1e-12)


def test_dimer_thermo_closed_form():
    """s=1/2 dimer: levels -3/4 (singlet) and 1/4 (triplet); chi = 2 beta e^{-beta/4} / Z (g = 1)."""
    T = np.geomspace(0.05, 50, 25)
    _, blocks = _exact_blocks("dimer", 1)
    lnZ, E, C, chi, E0 = thermo(blocks, T)
    b = 1 / T
    Z = np.exp(0.75 * b) + 3 * np.exp(-0.25 * b)
    Em = (-0.75 * np.exp(0.75 * b) + 0.75 * np.exp(-0.25 * b)) / Z
    E2 = (0.5625 * np.exp(0.75 * b) + 3 * 0.0625 * np.exp(-0.25 * b)) / Z
    assert np.isclose(E0, -0.75)
    assert np.allclose(lnZ, np.log(Z), rtol=1e-12)
    assert np.allclose(E, Em, rtol=1e-12, atol=1e-14)
    p = 3 * np.exp(-0.25 * b) / Z  # two levels one unit apart: variance p (1 - p)
    assert np.allclose(C, b * b * p * (1 - p), rtol=1e-10, atol=1e-300)
    assert np.allclose(E2 - Em ** 2, p * (1 - p), atol=1e-12)
    assert np.allclose(chi, 2 * b * np.exp(-0.25 * b) / Z, rtol=1e-12)


def test_high_temperature_curie_limit():
    """chi T / g^2 -> N s(s+1)/3 as T -> infinity, for stochastic FTLM too (sum rule)."""
    c = cluster("icosahedron")
    g = Group(c.gens, c.bonds)
    two_s, N = 1, 12
    blocks = []
    for two_M in range(0, N * two_s + 1, 2):
        sec = SectorBasis(g, two_s, two_M)
        for ir in range(len(g.irreps)):
            blk = BlockBasis(sec, ir).with_hamiltonian(c.bonds)
            if blk.dim == 0:
                continue
            R = 2
            V0 = start_vectors(blk.dim, R, 0, two_M * 100 + ir)
            al, be = zip(*[lanczos(blk.hv, V0[:, r], 10) for r in range(R)])
            blocks.append(dict(two_M=two_M, d_gamma=g.irreps[ir].dim, dim=blk.dim, R=R, alpha=al, beta=be))
    T = np.array([1e8])
    _, _, _, chi, _ = thermo(blocks, T, g=2.0)
    assert np.isclose(chi[0] * T[0] / 4, N * 0.5 * 1.5 / 3, rtol=1e-6)
