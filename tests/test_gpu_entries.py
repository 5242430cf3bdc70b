"""Entry tables (Section 3's two-phase design): the table path reproduces the search path bitwise.

The build pass is the search part of the packed H·v kernel and writes the flips
in the kernel's own order, so a table-mode H·v must equal the search-mode H·v
element by element in FP64, FP32 and FP16 storage, for every block shape, and
the entry count must equal the number of admissible flips (Eq. 3) counted from
the exported labels.  The search path itself is checked against the oracle in
test_gpu_packed.py.
"""
import numpy as np
import pytest

from gpu_common import ftlm, product_group, torch_cuda

pytestmark = pytest.mark.gpu

SETS = [("icosahedron", 1, 0), ("icosahedron", 3, 2), ("cuboctahedron", 2, 4), ("cuboctahedron", 4, 32),
        ("tetrahedron", 5, 2), ("square:4x4", 1, 2)]


def _count_flips(labels, bonds, two_s, bits):
    lab = labels.astype(np.uint64)
    mask = np.uint64((1 << bits) - 1)
    n = 0
    for i, j in bonds:
        ai = (lab >> np.uint64(bits * int(i))) & mask
        aj = (lab >> np.uint64(bits * int(j))) & mask
        n += int(np.count_nonzero((ai < two_s) & (aj > 0))) + int(np.count_nonzero((ai > 0) & (aj < two_s)))
    return n


@pytest.mark.parametrize("name,two_s,two_M", SETS)
def test_table_hv_equals_search_hv_bitwise(name, two_s, two_M):
    torch = torch_cuda()
    F = ftlm()
    g = product_group(name)
    info = F.ftlm_group_info(g)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    labels, _ = F.ftlm_sector_export(sec)
    bits = max(1, int(np.ceil(np.log2(two_s + 1))))
    bonds, _ = F.ftlm_group_bonds(g)
    full = all(d <= 5 for d in info["dims"]) and len(info["dims"]) <= 10
    sets = [F.ftlm_build_multiblock(sec, list(range(len(info["dims"]))))] if full else []
    sets += [F.ftlm_build_multiblock(sec, [k]) for k in range(len(info["dims"])) if info["dims"][k] <= 5][:3]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    cases = []
    for mb in sets:
        try:
            rows = F.ftlm_multiblock_packed_rows(mb)
        except F.FtlmError:
            continue
        for dt, tdt, B in ((F.F64, torch.float64, 3), (F.F32, torch.float32, 8), (F.F16, torch.float16, 8),
                           (F.F32, torch.float32, 1), (F.F64, torch.float64, 1), (F.F16, torch.float16, 1)):
            x = torch.randn((rows, B), device="cuda", generator=gen).to(tdt)
            y = torch.full_like(x, float("nan"))
            F.ftlm_hv_packed(mb, dt, B, x, y)
            cases.append((mb, dt, B, x, y))
    assert cases
    n = F.ftlm_sector_build_entries(sec)
    assert n == _count_flips(labels, bonds, two_s, bits)
    for mb, dt, B, x, y in cases:
        y2 = torch.full_like(x, float("nan"))
        F.ftlm_hv_packed(mb, dt, B, x, y2)
        F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
        if B == 1 and F.ftlm_multiblock_info(mb)["n_blocks"] == 1:
            # one thread per representative: the same terms summed in entry order, equal to rounding
            tol = {F.F64: 1e-13, F.F32: 3e-6, F.F16: 2e-3}[dt]
            scale = float(y.double().abs().max()) + 1.0
            assert float((y.double() - y2.double()).abs().max()) <= tol * scale, (dt, B)
        else:
            assert torch.equal(y, y2), (dt, B)
    F.ftlm_sector_free_entries(sec)
    mb, dt, B, x, y = cases[0]
    y3 = torch.full_like(x, float("nan"))
    F.ftlm_hv_packed(mb, dt, B, x, y3)
    assert torch.equal(y, y3)


def test_table_lanczos_matches_search_lanczos():
    torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")
    sec = F.ftlm_build_sector(g, 3, 4)
    mb = F.ftlm_build_multiblock(sec, list(range(10)))
    ids = list(range(10))
    a0, b0, s0 = F.ftlm_lanczos_multi(mb, F.F64, 4, 30, 9, ids, F.GAUSS)
    F.ftlm_sector_build_entries(sec)
    a1, b1, s1 = F.ftlm_lanczos_multi(mb, F.F64, 4, 30, 9, ids, F.GAUSS)
    assert np.array_equal(s0, s1)
    assert np.allclose(a0, a1, rtol=1e-12, atol=1e-12) and np.allclose(b0, b1, rtol=1e-12, atol=1e-12)


def test_table_hv_full_size_icosidodecahedron():
    """The benchmark sector (1.3e6 representatives, 4.0e7 flips): table and search paths agree bitwise."""
    torch = torch_cuda()
    F = ftlm()
    g = product_group("icosidodecahedron")
    sec = F.ftlm_build_sector(g, 1, 0)
    mb = F.ftlm_build_multiblock(sec, list(range(10)))
    rows = F.ftlm_multiblock_packed_rows(mb)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    x = torch.randn((rows, 8), device="cuda", generator=gen)
    y = torch.empty_like(x)
    F.ftlm_hv_packed(mb, F.F32, 8, x, y)
    n = F.ftlm_sector_build_entries(sec)
    assert 3.9e7 < n < 4.1e7
    y2 = torch.empty_like(x)
    F.ftlm_hv_packed(mb, F.F32, 8, x, y2)
    F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
    assert torch.equal(y, y2)


def test_table_lanczos_one_block_one_chain():
    """K = 1, B = 1 (the one-thread-per-representative table kernel): the Lanczos coefficients match
    the search path's in FP64 to rounding."""
    torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")
    sec = F.ftlm_build_sector(g, 3, 2)
    for ir in (0, 6, 9):
        blk = F.ftlm_build_block(sec, ir)
        F.ftlm_sector_free_entries(sec)
        a0, b0, s0 = F.ftlm_lanczos(blk, F.F64, 1, 30, 3, ir)
        F.ftlm_sector_build_entries(sec)
        a1, b1, s1 = F.ftlm_lanczos(blk, F.F64, 1, 30, 3, ir)
        assert np.array_equal(s0, s1)
        assert np.allclose(a0, a1, rtol=1e-11, atol=1e-11) and np.allclose(b0, b1, rtol=1e-11, atol=1e-11)


def test_lane_kernel_several_parts():
    """The one-thread-per-representative kernel with several parts in one launch (every M >= 0 sector of
    a cluster as single-block sets at R = 1, each sector with its entry table): every set's coefficients
    match the same set run alone on the search path, to rounding (FP64)."""
    torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")
    ir = 8  # a five-dimensional irrep
    sets, secs, ids = [], [], []
    for two_M in range(0, 14, 2):
        sec = F.ftlm_build_sector(g, 3, two_M)
        mb = F.ftlm_build_multiblock(sec, [ir])
        if F.ftlm_multiblock_info(mb)["dims"][0] < 40:
            continue
        sets.append(mb)
        secs.append(sec)
        ids.append([64 * two_M + ir])
    assert len(sets) >= 4
    alone = []
    for mb, bid in zip(sets, ids):
        a0, b0, s0 = F.ftlm_lanczos_multi(mb, F.F64, 1, 25, 9, bid, F.GAUSS)
        alone.append((a0, b0, s0))
    for sec in secs:
        F.ftlm_sector_build_entries(sec)
    a, b, st = F.ftlm_lanczos_sets(sets, F.F64, 1, 25, 9, ids, F.GAUSS)
    for i, (a0, b0, s0) in enumerate(alone):
        assert np.array_equal(st[i], s0)
        k = int(s0[0, 0])
        scale = np.abs(a0[0, 0, :k]).max() + 1.0
        assert np.abs(a[i, 0, 0, :k] - a0[0, 0, :k]).max() <= 1e-10 * scale
        assert np.abs(b[i, 0, 0, :k] - b0[0, 0, :k]).max() <= 1e-10 * scale
