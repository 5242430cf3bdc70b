"""GPU Lanczos, tridiagonal eigensolve and thermal sums vs the oracle (Section 2.2, Eqs. 4-7, 14).

Config "icosahedron s=1/2": all M >= 0 sectors x all 10 irreps, R = 4 Gaussian
start vectors (seed 0), 30 Lanczos steps, 200 log-spaced T in [0.02, 100].
block_id of block (M, Gamma) = 64 * 2M + Gamma.
"""
import numpy as np
import pytest
import scipy.linalg

from gpu_common import ftlm, product_group
from helpers import oracle_group
from oracle.basis import BlockBasis, SectorBasis
from oracle.lanczos import lanczos, start_vectors, thermo
from workloads import cluster

pytestmark = pytest.mark.gpu

T_GRID = 0.02 * 5000.0 ** (np.arange(200) / 199.0)


def test_ritz_matches_lapack():
    F = ftlm()
    rng = np.random.default_rng(3)
    n, ld = 40, 60
    m = rng.integers(1, ld + 1, n).astype(np.int32)
    a = rng.standard_normal((n, ld))
    b = np.abs(rng.standard_normal((n, ld))) + 0.1
    th, w = F.ftlm_ritz(a, b, m)
    for c in range(n):
        k = m[c]
        if k == 1:
            ev, z0 = a[c, :1], np.ones(1)
        else:
            ev, Z = scipy.linalg.eigh_tridiagonal(a[c, :k], b[c, :k - 1])
            z0 = Z[0] ** 2
        assert np.allclose(th[c, :k], ev, atol=1e-12 * (1 + np.abs(ev).max()))
        assert abs(w[c, :k].sum() - 1) < 1e-12
        for p in range(4):
            assert np.isclose((w[c, :k] * th[c, :k] ** p).sum(), (z0 * ev ** p).sum(), rtol=1e-10, atol=1e-10)
        assert np.all(th[c, k:] == 0)


def _config1_blocks(dtype_gpu=None, R=4, n_steps=30, seed=0, with_oracle=True):
    F = ftlm()
    name, two_s = "icosahedron", 1
    g = product_group(name)
    og = oracle_group(name)
    c = cluster(name)
    gpu_blocks, ora_blocks = [], []
    for two_M in range(0, 13, 2):
        sec = F.ftlm_build_sector(g, two_s, two_M)
        osec = SectorBasis(og, two_s, two_M) if with_oracle else None
        for ir, irr in enumerate(og.irreps):
            blk = F.ftlm_build_block(sec, ir)
            dim = F.ftlm_basis_info(blk)["dim"]
            if dim == 0:
                continue
            bid = 64 * two_M + ir
            if dtype_gpu is not None:
                a, b, st = F.ftlm_lanczos(blk, dtype_gpu, R, n_steps, seed, bid)
                gpu_blocks.append(dict(two_M=two_M, d_gamma=irr.dim, dim=dim, alpha=a, beta=b, steps=st))
            if with_oracle:
                ob = BlockBasis(osec, ir).with_hamiltonian(c.bonds)
                V0 = start_vectors(dim, R, seed, bid)
                al, be = zip(*[lanczos(ob.hv, V0[:, r], n_steps) for r in range(R)])
                ora_blocks.append(dict(two_M=two_M, d_gamma=irr.dim, dim=dim, R=R, alpha=al, beta=be))
    return gpu_blocks, ora_blocks


def test_start_vectors_match_oracle_philox():
    """First Lanczos coefficient alpha_0 = <v0|H|v0> needs the same start vector on both sides."""
    F = ftlm()
    g = product_group("icosahedron")
    og = oracle_group("icosahedron")
    c = cluster("icosahedron")
    for rng_name, rng in (("gauss", F.GAUSS), ("rademacher", F.RADEMACHER)):
        blk = F.ftlm_build_basis(g, 3, 0, 8)
        dim = F.ftlm_basis_info(blk)["dim"]
        a, b, st = F.ftlm_lanczos(blk, F.F64, 3, 2, 11, 77, rng)
        ob = BlockBasis(SectorBasis(og, 3, 0), 8).with_hamiltonian(c.bonds)
        V0 = start_vectors(dim, 3, 11, 77, rng=rng_name)
        for r in range(3):
            ar, br = lanczos(ob.hv, V0[:, r], 2)
            assert np.allclose(a[r, :2], ar, rtol=1e-12, atol=1e-12)
            assert np.allclose(b[r, :2], br, rtol=1e-12, atol=1e-12)


def test_lanczos_f64_coefficients_match_oracle():
    """Per-step alpha/beta agree before orthogonality is lost (large block, 12 steps)."""
    F = ftlm()
    g = product_group("icosahedron")
    og = oracle_group("icosahedron")
    c = cluster("icosahedron")
    blk = F.ftlm_build_basis(g, 3, 0, 9)
    dim = F.ftlm_basis_info(blk)["dim"]
    a, b, st = F.ftlm_lanczos(blk, F.F64, 5, 12, 4, 9)
    ob = BlockBasis(SectorBasis(og, 3, 0), 9).with_hamiltonian(c.bonds)
    V0 = start_vectors(dim, 5, 4, 9)
    for r in range(5):
        ar, br = lanczos(ob.hv, V0[:, r], 12)
        assert st[r] == len(ar) == 12
        assert np.allclose(a[r], ar, rtol=1e-10, atol=1e-10)
        assert np.allclose(b[r], br, rtol=1e-10, atol=1e-10)


def test_thermo_matches_oracle_on_same_coefficients():
    F = ftlm()
    _, ora = _config1_blocks(None)
    blocks = []
    for bl in ora:
        R = bl["R"]
        ld = 30
        A = np.zeros((R, ld))
        Bt = np.zeros((R, ld))
        st = np.zeros(R, dtype=np.int32)
        for r in range(R):
            m = len(bl["alpha"][r])
            A[r, :m], Bt[r, :m], st[r] = bl["alpha"][r], bl["beta"][r], m
        blocks.append(dict(two_M=bl["two_M"], d_gamma=bl["d_gamma"], dim=bl["dim"], alpha=A, beta=Bt, steps=st))
    lnZ, E, C, chi, E0 = F.ftlm_thermo(blocks, T_GRID, g=2.0)
    rl, rE, rC, rchi, rE0 = thermo(ora, T_GRID, g=2.0)
    assert abs(E0 - rE0) < 1e-12 * abs(rE0)
    assert np.allclose(lnZ, rl, rtol=1e-12)
    assert np.abs(E - rE).max() < 1e-11 * np.abs(rE).max()
    assert np.abs(C - rC).max() < 1e-11 * rC.max()
    assert np.abs(chi - rchi).max() < 1e-11 * rchi.max()


def test_config1_pipeline_f64_matches_oracle():
    """Whole FTLM of the s=1/2 icosahedron on the GPU in FP64 vs the oracle: 1e-10 relative."""
    F = ftlm()
    gpu, ora = _config1_blocks(F.F64)
    lnZ, E, C, chi, E0 = F.ftlm_thermo(gpu, T_GRID)
    rl, rE, rC, rchi, rE0 = thermo(ora, T_GRID)
    for gb, ob in zip(gpu, ora):
        assert [int(s) for s in gb["steps"]] == [len(a) for a in ob["alpha"]]
    assert abs(E0 - rE0) <= 1e-10 * abs(rE0)
    assert np.allclose(lnZ, rl, rtol=1e-10)
    assert np.abs(C - rC).max() <= 1e-10 * rC.max()
    assert np.abs(chi - rchi).max() <= 1e-10 * rchi.max()
    assert np.abs(E - rE).max() <= 1e-10 * np.abs(rE).max()
    # Curie limit (Section 4.1): T chi -> N s(s+1)/3 at high T
    _, _, _, chi_hi, _ = F.ftlm_thermo(gpu, np.array([1e9]))
    assert abs(chi_hi[0] * 1e9 - 12 * 0.75 / 3) < 1e-6


def test_config1_mixed_precision_error():
    """FP32 vectors with FP64 alpha/beta: E0 within 1e-5, C and chi within 1e-4 of their maxima (T >= 0.05)."""
    F = ftlm()
    g64, _ = _config1_blocks(F.F64, with_oracle=False)
    g32, _ = _config1_blocks(F.F32, with_oracle=False)
    a = F.ftlm_thermo(g64, T_GRID)
    b = F.ftlm_thermo(g32, T_GRID)
    sel = T_GRID >= 0.05
    assert abs(a[4] - b[4]) <= 1e-5 * abs(a[4])
    assert np.abs(a[2] - b[2])[sel].max() <= 1e-4 * a[2].max()
    assert np.abs(a[3] - b[3])[sel].max() <= 1e-4 * a[3].max()
