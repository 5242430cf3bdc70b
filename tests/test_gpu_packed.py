"""Packed multi-block H·v (every irrep block of a sector in one launch, Eqs. 15-16) vs the oracle.

The packed layout interleaves the rows of all blocks by representative; the
per-block results are recovered with ftlm_multiblock_unpack and compared with
the oracle's BlockBasis.hv block by block.  Also: the pack/unpack round trip,
the bulk-copy and lane-copy gather paths, the bounded-wait timeout status, and
the full-size s=1/2 icosidodecahedron M=0 sector on sampled rows.
"""
import os

import numpy as np
import pytest

from gpu_common import ftlm, product_group, torch_cuda
from helpers import oracle_group
from oracle import native
from oracle.basis import BlockBasis, SectorBasis, hv_rows_by_label
from workloads import cluster, label_keyed_values, rand_block_vectors

pytestmark = pytest.mark.gpu

# full irrep sets of I_h (10 blocks), O_h (10) and T_d (5); s = 1/2 (32-bit labels) and larger s
SETS = [("icosahedron", 1, 0), ("icosahedron", 1, 4), ("icosahedron", 3, 2), ("cuboctahedron", 1, 0),
        ("cuboctahedron", 2, 4), ("cuboctahedron", 4, 32), ("tetrahedron", 5, 2), ("tetrahedron", 1, 0)]

_SECTORS = {}


def _oracle_sector(name, two_s, two_M):
    key = (name, two_s, two_M)
    if key not in _SECTORS:
        _SECTORS[key] = SectorBasis(oracle_group(name), two_s, two_M)
    return _SECTORS[key]


def _setup(name, two_s, two_M):
    F = ftlm()
    g = product_group(name)
    og = oracle_group(name)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    mb = F.ftlm_build_multiblock(sec, list(range(len(og.irreps))))
    return F, og, sec, mb


def _packed_hv(F, torch, mb, dims, xs_np, B, dtype):
    tdt = torch.float64 if dtype == F.F64 else torch.float32
    rows = F.ftlm_multiblock_packed_rows(mb)
    xs = [torch.from_numpy(np.ascontiguousarray(x)).to("cuda", tdt) for x in xs_np]
    xp = torch.full((rows, B), float("nan"), dtype=tdt, device="cuda")
    F.ftlm_multiblock_pack(mb, dtype, B, xs, xp)
    yp = torch.full_like(xp, float("nan"))
    F.ftlm_hv_packed(mb, dtype, B, xp, yp)
    F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
    ys = [torch.full((d, B), float("nan"), dtype=tdt, device="cuda") for d in dims]
    F.ftlm_multiblock_unpack(mb, dtype, B, yp, ys)
    return [y.double().cpu().numpy() for y in ys], xp, yp


@pytest.mark.parametrize("name,two_s,two_M", SETS)
@pytest.mark.parametrize("B", [1, 3, 8, 24])
def test_packed_hv_matches_oracle(name, two_s, two_M, B):
    torch = torch_cuda()
    F, og, sec, mb = _setup(name, two_s, two_M)
    c = cluster(name)
    dims = F.ftlm_multiblock_info(mb)["dims"]
    osec = _oracle_sector(name, two_s, two_M)
    xs = [rand_block_vectors(d, B, seed=31 * k + B) for k, d in enumerate(dims)]
    refs = [BlockBasis(osec, k).with_hamiltonian(c.bonds).hv(x) if d else None for k, (d, x) in
            enumerate(zip(dims, xs))]
    for dtype, tol in ((F.F64, 1e-13), (F.F32, 3e-6)):
        ys, _, _ = _packed_hv(F, torch, mb, dims, xs, B, dtype)
        for k in range(len(dims)):
            if dims[k] == 0:
                continue
            scale = np.abs(refs[k]).max() + 1e-300
            assert np.abs(ys[k] - refs[k]).max() <= tol * scale, (k, dtype)


def test_pack_unpack_round_trip_is_exact():
    torch = torch_cuda()
    F, og, sec, mb = _setup("icosahedron", 3, 0)
    dims = F.ftlm_multiblock_info(mb)["dims"]
    rows = F.ftlm_multiblock_packed_rows(mb)
    n_reps = F.ftlm_sector_info(sec)["n_reps"]
    assert rows == n_reps * sum(ir.dim for ir in og.irreps)
    xs = [torch.from_numpy(rand_block_vectors(d, 5, seed=k)).cuda() for k, d in enumerate(dims)]
    xp = torch.full((rows, 5), float("nan"), dtype=torch.float64, device="cuda")
    F.ftlm_multiblock_pack(mb, F.F64, 5, xs, xp)
    assert torch.isfinite(xp).all()
    # the lift is an isometry: squared norms agree block by block
    assert abs(float((xp * xp).sum()) - sum(float((x * x).sum()) for x in xs)) <= 1e-12 * float((xp * xp).sum())
    back = [torch.zeros_like(x) for x in xs]
    F.ftlm_multiblock_unpack(mb, F.F64, 5, xp, back)
    for a, b in zip(xs, back):
        assert float((a - b).abs().max()) <= 1e-14 * (float(a.abs().max()) + 1e-300)


def test_bulk_copy_and_lane_copy_gathers_agree_bitwise():
    torch = torch_cuda()
    F, og, sec, mb = _setup("icosahedron", 1, 2)
    dims = F.ftlm_multiblock_info(mb)["dims"]
    xs = [rand_block_vectors(d, 8, seed=k) for k, d in enumerate(dims)]
    for dtype in (F.F32, F.F64):
        _, _, y_tma = _packed_hv(F, torch, mb, dims, xs, 8, dtype)
        os.environ["FTLM_HV_GATHER"] = "direct"
        try:
            _, _, y_dir = _packed_hv(F, torch, mb, dims, xs, 8, dtype)
        finally:
            del os.environ["FTLM_HV_GATHER"]
        assert torch.equal(y_tma, y_dir)


def test_bounded_wait_timeout_is_reported_and_context_survives():
    """A one-cycle wait budget runs out on the first bulk-copy wait of a warp whose gathers come from DRAM
    (the full-size icosidodecahedron M=0 sector, 1.3 GB packed vector, beyond L2): the kernel drains its
    copies and returns, ftlm_basis_check reports FTLM_ETIMEOUT, the error word is cleared, and the next call
    with the default budget is bitwise the same as before."""
    torch = torch_cuda()
    F = ftlm()
    g = product_group("icosidodecahedron")
    sec = F.ftlm_build_sector(g, 1, 0)
    mb = F.ftlm_build_multiblock(sec, list(range(10)))
    rows = F.ftlm_multiblock_packed_rows(mb)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    xp = torch.randn((rows, 8), dtype=torch.float32, device="cuda", generator=gen)
    y_ref = torch.empty_like(xp)
    F.ftlm_hv_packed(mb, F.F32, 8, xp, y_ref)
    blk0 = F.ftlm_multiblock_block(mb, 0)
    F.ftlm_basis_check(blk0)
    yp = torch.zeros_like(xp)
    F.ftlm_set_wait_limit(1)
    try:
        F.ftlm_hv_packed(mb, F.F32, 8, xp, yp)
        with pytest.raises(F.FtlmError) as e:
            F.ftlm_basis_check(blk0)
        assert e.value.status == F.ETIMEOUT
    finally:
        F.ftlm_set_wait_limit(0)
    F.ftlm_basis_check(blk0)  # the error word was cleared
    F.ftlm_hv_packed(mb, F.F32, 8, xp, yp)
    F.ftlm_basis_check(blk0)
    assert torch.equal(yp, y_ref)


def _block_x_from_labels(labels, ng, off, B, seed):
    """Block vector whose rows depend only on (representative label, k, b): label-keyed inputs."""
    dmax = max(1, int(ng.max()) if len(ng) else 1)
    vals = label_keyed_values(labels, dmax, B, seed)
    keep = np.arange(dmax)[None, :] < ng[:, None].astype(np.int64)
    X = vals[keep]
    assert X.shape[0] == int(off[-1])
    return X


@pytest.mark.parametrize("dtype_name", ["f32", "f64"])
def test_icosidodecahedron_m0_all_irreps_packed_and_multi_sampled_rows(dtype_name):
    """Full-size s=1/2 icosidodecahedron M=0 sector, all 10 irreps, B = 8 (the benchmark's launch): the packed
    H·v and the per-block multi-block H·v against the label-keyed oracle on sampled rows of every block."""
    torch = torch_cuda()
    F = ftlm()
    name, two_s, two_M, B = "icosidodecahedron", 1, 0, 8
    og = oracle_group(name)
    c = cluster(name)
    g = product_group(name)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    mb = F.ftlm_build_multiblock(sec, list(range(10)))
    dims = F.ftlm_multiblock_info(mb)["dims"]
    dtype, tdt, tol = ((F.F64, torch.float64, 1e-12) if dtype_name == "f64" else (F.F32, torch.float32, 2e-5))
    rng = np.random.default_rng(17)
    sample = set()
    while len(sample) < 40:
        bits = rng.permutation(np.r_[np.ones(15, dtype=np.int64), np.zeros(15, dtype=np.int64)])
        lab = int(sum(int(v) << k for k, v in enumerate(bits)))
        sample.add(native.min_rep(og.n_sites, 2, og.perms, lab)[0])
    sample = sorted(sample)
    xs, exports = [], []
    for k in range(10):
        labels, _, ng, off = F.ftlm_basis_export(F.ftlm_multiblock_block(mb, k))
        exports.append((labels, ng, off))
        xs.append(torch.from_numpy(_block_x_from_labels(labels, ng, off, B, 100 + k)).to("cuda", tdt))
    rows = F.ftlm_multiblock_packed_rows(mb)
    xp = torch.empty((rows, B), dtype=tdt, device="cuda")
    F.ftlm_multiblock_pack(mb, dtype, B, xs, xp)
    yp = torch.empty_like(xp)
    F.ftlm_hv_packed(mb, dtype, B, xp, yp)
    F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
    del xp
    ys_packed = [torch.empty_like(x) for x in xs]
    F.ftlm_multiblock_unpack(mb, dtype, B, yp, ys_packed)
    del yp
    ys_multi = [torch.empty_like(x) for x in xs]
    F.ftlm_hv_multi(mb, dtype, B, xs, ys_multi)
    F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
    for k in range(10):
        labels, ng, off = exports[k]
        rows_ref = hv_rows_by_label(og, k, c.bonds, 1.0, two_s, sample,
                                    lambda lab, n, s=100 + k: label_keyed_values([lab], n, B, s)[0])
        pos = np.searchsorted(labels, np.array(sample, dtype=np.uint64))
        for Y in (ys_packed[k].double().cpu().numpy(), ys_multi[k].double().cpu().numpy()):
            scale = np.abs(Y).max()
            for lab, p, yr in zip(sample, pos, rows_ref):
                assert labels[p] == lab
                if yr is None:
                    assert ng[p] == 0
                    continue
                got = Y[int(off[p]):int(off[p]) + int(ng[p])]
                assert np.abs(got - yr).max() <= tol * scale


@pytest.mark.parametrize("name,two_s", [("icosahedron", 3), ("cuboctahedron", 2)])
def test_lanczos_sets_matches_each_set_alone(name, two_s):
    """Every M >= 0 sector of a cluster as the parts of one launch per kernel (ftlm_lanczos_sets) gives each
    sector's coefficients of ftlm_lanczos_multi on that sector alone (FP64, Rademacher, R = 5 chains)."""
    F = ftlm()
    g = product_group(name)
    n_ir = len(oracle_group(name).irreps)
    n_sites = oracle_group(name).n_sites
    sets, ids = [], []
    for two_M in range(0, n_sites * two_s + 1, 2 * max(1, n_sites * two_s // 8)):
        sec = F.ftlm_build_sector(g, two_s, two_M)
        sets.append(F.ftlm_build_multiblock(sec, list(range(n_ir))))
        ids.append([64 * two_M + k for k in range(n_ir)])
    a, b, st = F.ftlm_lanczos_sets(sets, F.F64, 5, 20, 7, ids, F.RADEMACHER)
    for i, mb in enumerate(sets):
        a1, b1, s1 = F.ftlm_lanczos_multi(mb, F.F64, 5, 20, 7, ids[i], F.RADEMACHER)
        assert np.array_equal(st[i], s1)
        assert np.allclose(a[i], a1, rtol=1e-10, atol=1e-11)
        assert np.allclose(b[i], b1, rtol=1e-10, atol=1e-11)


def test_autotune_changes_timing_only():
    """The autotuner tries geometries on the plan's own vectors and keeps the fastest; every candidate
    computes identical rows (one warp per representative, fixed flip order), so H·v is bitwise unchanged
    and Lanczos coefficients agree to rounding."""
    torch = torch_cuda()
    F, og, sec, mb = _setup("icosahedron", 3, 2)
    rows = F.ftlm_multiblock_packed_rows(mb)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    xp = torch.randn((rows, 8), dtype=torch.float32, device="cuda", generator=gen)
    y0 = torch.empty_like(xp)
    F.ftlm_hv_packed(mb, F.F32, 8, xp, y0)
    a0, b0, s0 = F.ftlm_lanczos_multi(mb, F.F64, 4, 12, 3, list(range(10)))
    F.ftlm_set_autotune(-1)
    F.ftlm_set_autotune(1)
    try:
        y1 = torch.empty_like(xp)
        F.ftlm_hv_packed(mb, F.F32, 8, xp, y1)
        F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
        a1, b1, s1 = F.ftlm_lanczos_multi(mb, F.F64, 4, 12, 3, list(range(10)))
        report = F.ftlm_autotune_report()
    finally:
        F.ftlm_set_autotune(-1)
        F.ftlm_set_autotune(0)
    assert torch.equal(y0, y1)
    assert np.array_equal(s0, s1)
    assert np.allclose(a0, a1, rtol=1e-11, atol=1e-12) and np.allclose(b0, b1, rtol=1e-11, atol=1e-12)
    assert "tried=" in report and len(report.strip().splitlines()) >= 2
