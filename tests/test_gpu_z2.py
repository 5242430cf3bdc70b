"""Spin-flip sectors (G x Z_2 at M = 0, Section 2.2) on the GPU vs the oracle.

The oracle's extension (oracle.group.SpinFlipExtended) is pinned on the CPU by the
dense projector check, the flip parity of the Eq. 12 vectors and the spectrum union
(tests/test_oracle_z2.py).  Here: representatives, 256-bit stabilizers and n_Gamma+-
bit-exact; H·v of single Gamma+- blocks and of the all-Gamma+ / all-Gamma- packed sets
against the oracle's block H·v (FP64 1e-12, FP32 3e-6); the entry table reproducing the
search path bitwise; and exact Lanczos spectra whose Gamma+ and Gamma- union is the
plain sector's Gamma spectrum.
"""
import numpy as np
import pytest

from gpu_common import ftlm, product_group, torch_cuda
from helpers import oracle_group
from oracle.basis import BlockBasis, SectorBasis
from oracle.group import SpinFlipExtended
from workloads import cluster, rand_block_vectors

pytestmark = pytest.mark.gpu

CASES = [("icosahedron", 1), ("icosahedron", 3), ("cuboctahedron", 2), ("tetrahedron", 2), ("ring:6", 2),
         ("square:4x4", 1), ("chain:8", 1), ("q8", 2), ("complete:7", 2), ("petersen", 1)]


@pytest.mark.parametrize("name,two_s", CASES)
def test_flip_sector_matches_oracle(name, two_s):
    torch = torch_cuda()
    F = ftlm()
    g = product_group(name)
    og = oracle_group(name)
    gx = SpinFlipExtended(og)
    c = cluster(name)
    sec = F.ftlm_build_sector_flip(g, two_s)
    sym = F.ftlm_sector_symmetry(sec)
    assert sym == dict(order=2 * og.order, n_irreps=2 * len(og.irreps), flip=1)
    osec = SectorBasis(gx, two_s, 0)
    labels, masks = F.ftlm_sector_export(sec)
    bits = max(1, int(np.ceil(np.log2(two_s + 1))))
    d = two_s + 1
    # packed labels -> base-d labels (the oracle's encoding, Eq. 2)
    base = np.zeros(len(labels), dtype=np.uint64)
    for k in reversed(range(c.n_sites)):
        base = base * np.uint64(d) + ((labels >> np.uint64(bits * k)) & np.uint64((1 << bits) - 1))
    order = np.argsort(base)
    assert np.array_equal(base[order], osec.reps.astype(np.uint64))
    W = osec.stab.shape[1]
    assert np.array_equal(masks[order][:, :W], osec.stab.astype(np.uint64))
    rng = np.random.default_rng(2)
    for k, ir in enumerate(gx.irreps):
        if ir.rho is None:
            continue
        ob = BlockBasis(osec, k).with_hamiltonian(c.bonds)
        blk = F.ftlm_build_block(sec, k)
        _, _, ng, _ = F.ftlm_basis_export(blk)
        assert np.array_equal(ng[order], ob.n.astype(np.uint8))
        assert F.ftlm_basis_info(blk)["dim"] == ob.dim
        if ob.dim == 0 or (labels[order] != labels).any():
            continue  # the GPU rows follow the packed-label order; compared only when it is the oracle's
        x = rng.standard_normal((ob.dim, 3))
        y_ref = ob.hv(x)
        for dt, tdt, tol in ((F.F64, torch.float64, 1e-12), (F.F32, torch.float32, 3e-6)):
            xt = torch.tensor(x, dtype=tdt, device="cuda")
            yt = torch.full_like(xt, float("nan"))
            F.ftlm_hv(blk, dt, 3, xt, yt)
            F.ftlm_basis_check(blk)
            scale = np.abs(y_ref).max() + 1.0
            assert np.abs(yt.double().cpu().numpy() - y_ref).max() <= tol * scale, (k, dt)


def test_flip_packed_sets_and_entry_table():
    torch = torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")
    og = oracle_group("icosahedron")
    gx = SpinFlipExtended(og)
    c = cluster("icosahedron")
    sec = F.ftlm_build_sector_flip(g, 3)
    osec = SectorBasis(gx, 3, 0)
    n_ir = len(og.irreps)
    outs = {}
    for par in (0, 1):  # all Gamma+ blocks, all Gamma- blocks: the I_h packed shape with signs
        irreps = [2 * i + par for i in range(n_ir)]
        mb = F.ftlm_build_multiblock(sec, irreps)
        dims = F.ftlm_multiblock_info(mb)["dims"]
        obs = [BlockBasis(osec, k).with_hamiltonian(c.bonds) for k in irreps]
        assert dims == [ob.dim for ob in obs]
        B = 8
        xs = [rand_block_vectors(dd, B, seed=7 + 10 * i + par) for i, dd in enumerate(dims)]
        xt = [torch.tensor(x, device="cuda") for x in xs]
        rows = F.ftlm_multiblock_packed_rows(mb)
        xp = torch.full((rows, B), float("nan"), dtype=torch.float64, device="cuda")
        F.ftlm_multiblock_pack(mb, F.F64, B, xt, xp)
        yp = torch.full_like(xp, float("nan"))
        F.ftlm_hv_packed(mb, F.F64, B, xp, yp)
        F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
        ys = [torch.full((d, B), float("nan"), dtype=torch.float64, device="cuda") for d in dims]
        F.ftlm_multiblock_unpack(mb, F.F64, B, yp, ys)
        for ob, x, y in zip(obs, xs, ys):
            if ob.dim:
                ref = ob.hv(x)
                assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * (np.abs(ref).max() + 1.0)
        outs[par] = (mb, xp, yp)
    F.ftlm_sector_build_entries(sec)
    for par, (mb, xp, yp) in outs.items():
        y2 = torch.full_like(xp, float("nan"))
        F.ftlm_hv_packed(mb, F.F64, 8, xp, y2)
        assert torch.equal(yp, y2)


def test_flip_spectra_union_is_the_parent_spectrum():
    """Dense blocks from the GPU H·v on unit vectors: the Gamma+ and Gamma- spectra together are the
    plain M = 0 Gamma spectrum, level by level with multiplicities."""
    torch = torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")

    def dense(blk):
        dim = F.ftlm_basis_info(blk)["dim"]
        if dim == 0:
            return np.zeros(0)
        H = np.zeros((dim, dim))
        for c0 in range(0, dim, 32):
            B = min(32, dim - c0)
            x = torch.zeros((dim, B), dtype=torch.float64, device="cuda")
            x[c0:c0 + B] = torch.eye(B, dtype=torch.float64, device="cuda")
            y = torch.empty_like(x)
            F.ftlm_hv(blk, F.F64, B, x, y)
            H[:, c0:c0 + B] = y.cpu().numpy()
        F.ftlm_basis_check(blk)
        assert np.abs(H - H.T).max() < 1e-12
        return np.linalg.eigvalsh(H)

    checked = 0
    for two_s in (1, 2):
        plain = F.ftlm_build_sector(g, two_s, 0)
        flip = F.ftlm_build_sector_flip(g, two_s)
        for i in range(10):
            pb = F.ftlm_build_block(plain, i)
            if F.ftlm_basis_info(pb)["dim"] > 1200:
                continue
            ev = np.sort(np.concatenate([dense(F.ftlm_build_block(flip, k)) for k in (2 * i, 2 * i + 1)]))
            ref = dense(pb)
            assert len(ev) == len(ref) and np.abs(ev - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())
            checked += 1
    assert checked >= 12


def test_flip_sector_full_size_dodecahedron_block_dims():
    """The s=3/2 dodecahedron's M = 0 sector under G x Z_2 (3.6e8 representatives): every Gamma+-
    block dimension equals the oracle's character formula, and each pair adds up to Table 2."""
    torch_cuda()
    F = ftlm()
    from oracle.sector import block_dims

    g = product_group("dodecahedron")
    og = oracle_group("dodecahedron")
    ref = block_dims(SpinFlipExtended(og), 3, 0)
    sec = F.ftlm_build_sector_flip(g, 3)
    for k in range(2 * len(og.irreps)):
        blk = F.ftlm_build_block(sec, k)
        assert F.ftlm_basis_info(blk)["dim"] == ref[k], k
        del blk
