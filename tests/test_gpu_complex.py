"""Irreps of complex and quaternionic type (real forms) and dimensions 6..12 on the GPU vs the oracle.

The oracle's real forms are pinned on the CPU (tests/test_oracle_complex.py: dense projector
check, kappa-fold multiplets, weighted full-ED union, complete-graph closed form).  Here:
n_Gamma and block dimensions bit-exact; H·v of every block element by element (FP64 1e-13,
FP32 3e-6 of the largest output), on the search path and on the entry table (the warp kernels
bitwise equal to the search path, the one-thread-per-representative kernel to rounding); Lanczos
coefficients and the weighted thermal sums of a whole cluster against the oracle.
"""
import numpy as np
import pytest

from gpu_common import ftlm, product_group, torch_cuda
from helpers import oracle_group
from oracle.basis import BlockBasis, SectorBasis
from oracle.lanczos import lanczos, start_vectors, thermo
from workloads import cluster, rand_block_vectors

pytestmark = pytest.mark.gpu

# (cluster, 2s, 2M): C_n and T (complex pairs, d = 2), Q_8 (quaternionic, d = 4), AGL(1, 7) and
# AGL(1, 11) (d = 6 and 10 with complex pairs), S_5 on the Petersen graph (d = 4, 5, 6), the
# translations of the 4x4 torus; s = 1/2 (32-bit path) and general s (64-bit path)
CASES = [("chain:8", 1, 0), ("chain:7", 3, 1), ("tetrahedron:t", 3, 0), ("q8", 2, 0), ("q8", 3, 2),
         ("complete:7", 2, 0), ("complete:11", 1, 1), ("complete:11", 3, 1), ("petersen", 1, 0),
         ("petersen", 3, 2), ("square:4x4:t", 1, 0)]

_SECTORS = {}


def _oracle_sector(name, two_s, two_M):
    key = (name, two_s, two_M)
    if key not in _SECTORS:
        _SECTORS[key] = SectorBasis(oracle_group(name), two_s, two_M)
    return _SECTORS[key]


def _same_order(F, sec, osec, two_s, n_sites):
    """GPU labels are packed bit fields; rows line up with the oracle's when the orders agree."""
    labels, _ = F.ftlm_sector_export(sec)
    bits = max(1, int(np.ceil(np.log2(two_s + 1))))
    d = two_s + 1
    base = np.zeros(len(labels), dtype=np.uint64)
    for k in reversed(range(n_sites)):
        base = base * np.uint64(d) + ((labels >> np.uint64(bits * k)) & np.uint64((1 << bits) - 1))
    assert np.array_equal(np.sort(base), osec.reps.astype(np.uint64))
    return bool(np.array_equal(base, osec.reps.astype(np.uint64)))


@pytest.mark.parametrize("name,two_s,two_M", CASES)
def test_real_form_blocks_match_oracle(name, two_s, two_M):
    torch = torch_cuda()
    F = ftlm()
    g = product_group(name)
    og = oracle_group(name)
    c = cluster(name)
    info = F.ftlm_group_info(g)
    assert list(info["weights"]) == [ir.weight for ir in og.irreps]
    osec = _oracle_sector(name, two_s, two_M)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    assert _same_order(F, sec, osec, two_s, c.n_sites)
    checked = 0
    for ir, irr in enumerate(og.irreps):
        ob = BlockBasis(osec, ir).with_hamiltonian(c.bonds)
        blk = F.ftlm_build_block(sec, ir)
        _, _, ng, _ = F.ftlm_basis_export(blk)
        assert np.array_equal(ng, ob.n.astype(np.uint8))
        assert F.ftlm_basis_info(blk)["dim"] == ob.dim
        if ob.dim == 0:
            continue
        for dt, tdt, B, tol in ((F.F64, torch.float64, 1, 1e-13), (F.F64, torch.float64, 3, 1e-13),
                                (F.F32, torch.float32, 8, 3e-6)):
            x = rand_block_vectors(ob.dim, B, seed=100 * ir + B)
            y_ref = ob.hv(x)
            xd = torch.from_numpy(x).to("cuda", tdt).contiguous()
            yd = torch.full_like(xd, float("nan"))
            F.ftlm_hv(blk, dt, B, xd, yd)
            F.ftlm_basis_check(blk)
            err = np.abs(yd.double().cpu().numpy() - y_ref).max() / (np.abs(y_ref).max() + 1e-300)
            assert err < tol, (ir, irr.dim, irr.fs, dt, B, err)
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("name,two_s,two_M", [("petersen", 3, 2), ("complete:11", 3, 1), ("q8", 3, 2),
                                              ("square:4x4:t", 1, 0)])
def test_real_form_entry_table_paths(name, two_s, two_M):
    """Entry-table H·v of single blocks: B = 8 through the warp kernel (bitwise the search path);
    B = 1 through the one-thread-per-representative kernel (to rounding), FP64, FP32 and FP16."""
    torch = torch_cuda()
    F = ftlm()
    g = product_group(name)
    og = oracle_group(name)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    cases = []
    for ir in range(len(og.irreps)):
        mb = F.ftlm_build_multiblock(sec, [ir])
        rows = F.ftlm_multiblock_packed_rows(mb)
        if F.ftlm_multiblock_info(mb)["dims"][0] == 0:
            continue
        for dt, tdt, B in ((F.F64, torch.float64, 8), (F.F32, torch.float32, 8), (F.F64, torch.float64, 1),
                           (F.F32, torch.float32, 1), (F.F16, torch.float16, 1), (F.F16, torch.float16, 8)):
            x = torch.randn((rows, B), device="cuda", generator=gen).to(tdt)
            y = torch.full_like(x, float("nan"))
            F.ftlm_hv_packed(mb, dt, B, x, y)
            cases.append((mb, dt, B, x, y))
    F.ftlm_sector_build_entries(sec)
    for mb, dt, B, x, y in cases:
        y2 = torch.full_like(x, float("nan"))
        F.ftlm_hv_packed(mb, dt, B, x, y2)
        F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
        if B == 1:
            tol = {F.F64: 1e-13, F.F32: 3e-6, F.F16: 2e-3}[dt]
            scale = float(y.double().abs().max()) + 1.0
            assert float((y.double() - y2.double()).abs().max()) <= tol * scale, (dt, B)
        else:
            assert torch.equal(y, y2), (dt, B)


@pytest.mark.parametrize("name,two_s", [("q8", 2), ("chain:8", 1), ("complete:7", 2)])
def test_real_form_lanczos_and_thermo(name, two_s):
    """Every (M, Gamma) block of a cluster: FP64 Lanczos coefficients vs the oracle's (same Philox
    start vectors), then the weighted thermal sums (Eqs. 5-7, 14) vs the oracle's on the GPU's
    coefficients."""
    F = ftlm()
    g = product_group(name)
    og = oracle_group(name)
    c = cluster(name)
    N = c.n_sites
    R, n_steps, seed = 3, 12, 7
    T = 0.05 * 1000.0 ** (np.arange(60) / 59.0)
    gpu_blocks, ora_blocks = [], []
    for two_M in range(N * two_s % 2, N * two_s + 1, 2):
        sec = F.ftlm_build_sector(g, two_s, two_M)
        osec = SectorBasis(og, two_s, two_M)
        for ir, irr in enumerate(og.irreps):
            blk = F.ftlm_build_block(sec, ir)
            dim = F.ftlm_basis_info(blk)["dim"]
            if dim == 0:
                continue
            bid = 64 * two_M + ir
            a, b, st = F.ftlm_lanczos(blk, F.F64, R, n_steps, seed, bid)
            ob = BlockBasis(osec, ir).with_hamiltonian(c.bonds)
            V0 = start_vectors(dim, R, seed, bid)
            al, be = [], []
            for r in range(R):
                ar, br = lanczos(ob.hv, V0[:, r], n_steps)
                # a real-form block holds every level kappa times, so the Krylov space is exhausted after
                # dim / kappa steps at most; past a beta at rounding level the steps are rounding noise
                # and the two sides' stop tests may fire one step apart: compare the steps before it
                tiny = np.nonzero(np.abs(br) < 1e-8 * (np.abs(ar).max() + 1.0))[0]
                kk = len(ar) if len(tiny) == 0 else int(tiny[0]) + 1
                assert st[r] >= kk and (len(tiny) or st[r] == len(ar))
                assert np.allclose(a[r, :kk], ar[:kk], rtol=1e-10, atol=1e-10)
                assert np.allclose(b[r, :kk - 1], br[:kk - 1], rtol=1e-10, atol=1e-10)
                if len(tiny):  # the exhausting beta is at rounding level on both sides
                    assert abs(b[r, kk - 1]) < 1e-8 * (np.abs(ar).max() + 1.0)
                al.append(a[r, :st[r]])
                be.append(b[r, :st[r]])
            w = int(F.ftlm_group_info(g)["weights"][ir])
            assert w == irr.weight
            gpu_blocks.append(dict(two_M=two_M, d_gamma=w, dim=dim, alpha=a, beta=b, steps=st))
            ora_blocks.append(dict(two_M=two_M, d_gamma=w, dim=dim, R=R, alpha=al, beta=be))
    lnZ, E, C, chi, E0 = F.ftlm_thermo(gpu_blocks, T, 2.0)
    rl, rE, rC, rchi, rE0 = thermo(ora_blocks, T, g=2.0)
    assert abs(E0 - rE0) < 1e-10 * abs(rE0)
    assert np.allclose(lnZ, rl, rtol=1e-10)
    assert np.allclose(E, rE, rtol=1e-9, atol=1e-10)
    assert np.allclose(C, rC, rtol=1e-8, atol=1e-10)
    assert np.allclose(chi, rchi, rtol=1e-9, atol=1e-12)
