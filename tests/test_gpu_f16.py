"""FP16 vector storage (Section 3's half-precision mode, with Section 4.2's per-block power-of-two scale).

Reads widen FP16 to FP32, arithmetic is FP32 and every write rounds to nearest
FP16, so the FP16 H·v of an FP16 input is the FP32 H·v of the same values
rounded once: bitwise, in both gather paths.  The FP16 Lanczos run of a
cluster's blocks is compared with the FP64 run of the same seed through the
thermal sums (Eqs. 5-7, 14): the paper reports deviations of a few 1e-4 of the
curve maxima for C and chi and of the ground-state estimate; the bound here is
5e-3, with the measured values printed.
"""
import numpy as np
import pytest

from gpu_common import ftlm, product_group, torch_cuda

pytestmark = pytest.mark.gpu

T_GRID = 0.02 * 5000.0 ** (np.arange(200) / 199.0)


@pytest.mark.parametrize("name,two_s,two_M,B", [("icosahedron", 1, 0, 8), ("icosahedron", 3, 2, 3),
                                                ("cuboctahedron", 2, 4, 16), ("icosahedron", 1, 4, 1)])
def test_f16_hv_is_the_f32_hv_rounded_once(name, two_s, two_M, B):
    torch = torch_cuda()
    F = ftlm()
    g = product_group(name)
    n_ir = len(F.ftlm_group_info(g)["dims"])
    sec = F.ftlm_build_sector(g, two_s, two_M)
    mb = F.ftlm_build_multiblock(sec, list(range(n_ir)))
    rows = F.ftlm_multiblock_packed_rows(mb)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    x16 = torch.randn((rows, B), device="cuda", generator=gen).half()
    y16 = torch.full_like(x16, float("nan"))
    F.ftlm_hv_packed(mb, F.F16, B, x16, y16)
    F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
    x32 = x16.float()
    y32 = torch.full_like(x32, float("nan"))
    F.ftlm_hv_packed(mb, F.F32, B, x32, y32)
    assert torch.equal(y16, y32.half())


def _thermo_of_sets(F, g, two_s, dtype, R, n_steps, seed):
    info = F.ftlm_group_info(g)
    n_ir = len(info["dims"])
    N = info["n_sites"]
    sets, ids, Ms = [], [], []
    for two_M in range(N * two_s % 2, N * two_s + 1, 2):
        sec = F.ftlm_build_sector(g, two_s, two_M)
        sets.append(F.ftlm_build_multiblock(sec, list(range(n_ir))))
        ids.append([64 * two_M + k for k in range(n_ir)])
        Ms.append(two_M)
    a, b, st = F.ftlm_lanczos_sets(sets, dtype, R, n_steps, seed, ids, F.GAUSS)
    dims = [F.ftlm_multiblock_info(m)["dims"] for m in sets]
    blocks = [dict(two_M=Ms[i], d_gamma=int(info["dims"][k]), dim=dims[i][k], alpha=a[i][k], beta=b[i][k],
                   steps=st[i][k]) for i in range(len(sets)) for k in range(n_ir) if dims[i][k] > 0]
    return F.ftlm_thermo(blocks, T_GRID, 1.0)


def test_f16_lanczos_thermodynamics_within_storage_error():
    torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")
    ref = _thermo_of_sets(F, g, 3, F.F64, 8, 40, 2)
    got = _thermo_of_sets(F, g, 3, F.F16, 8, 40, 2)
    sel = T_GRID >= 0.05
    dE0 = abs(got[4] - ref[4]) / abs(ref[4])
    dC = np.abs(got[2] - ref[2])[sel].max() / ref[2][sel].max()
    dchi = np.abs(got[3] - ref[3])[sel].max() / ref[3][sel].max()
    print(f"FP16 vs FP64, s=3/2 icosahedron, R=8, 40 steps: dE0/E0 {dE0:.2e}, dC/Cmax {dC:.2e}, "
          f"dchi/chimax {dchi:.2e}")
    assert dE0 <= 5e-3 and dC <= 5e-3 and dchi <= 5e-3
    assert np.all(np.isfinite(got[0])) and np.all(np.isfinite(got[2]))


def test_f16_large_block_keeps_leading_coefficients():
    """A 6.5e6-row block: the scaled FP16 vectors keep the first Lanczos coefficients near FP64's."""
    torch_cuda()
    F = ftlm()
    g = product_group("icosidodecahedron")
    sec = F.ftlm_build_sector(g, 1, 0)
    blk = F.ftlm_build_block(sec, 9)  # H_u or H_g: d = 5
    a64, b64, s64 = F.ftlm_lanczos(blk, F.F64, 2, 12, 4, 9)
    a16, b16, s16 = F.ftlm_lanczos(blk, F.F16, 2, 12, 4, 9)
    assert np.array_equal(s64, s16)
    scale = np.abs(a64).max()
    assert np.abs(a16[:, :6] - a64[:, :6]).max() <= 1e-2 * scale
    assert np.abs(b16[:, :6] - b64[:, :6]).max() <= 1e-2 * scale
