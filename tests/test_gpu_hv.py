"""GPU H·v (Eqs. 15-16) vs the oracle, element by element, FP64 and FP32."""
import numpy as np
import pytest

from gpu_common import ftlm, product_group, torch_cuda
from helpers import oracle_group
from oracle import native
from oracle.basis import BlockBasis, SectorBasis, hv_rows_by_label
from workloads import cluster, label_keyed_values, rand_block_vectors

pytestmark = pytest.mark.gpu

# (cluster, 2s, 2M) covering s = 1/2 (32-bit XOR path) and general s (64-bit path),
# trivial and nontrivial stabilizers, d_Gamma = 1..5, ragged blocks
CASES = [("icosahedron", 1, 0), ("icosahedron", 1, 4), ("icosahedron", 3, 0), ("icosahedron", 3, 10),
         ("cuboctahedron", 1, 0), ("cuboctahedron", 2, 0), ("tetrahedron", 5, 2), ("ring:7", 1, 1),
         ("square:4x4", 1, 0), ("square:4x6", 1, 2), ("dodecahedron", 1, 0), ("ring:6", 5, 0),
         ("cuboctahedron", 4, 32),  # s = 2: 36-bit labels, most representatives above 2^32
         ("icosahedron", 5, 44)]  # s = 5/2: 3-bit fields, 36-bit labels

_SECTORS = {}


def _oracle_sector(name, two_s, two_M):
    key = (name, two_s, two_M)
    if key not in _SECTORS:
        _SECTORS[key] = SectorBasis(oracle_group(name), two_s, two_M)
    return _SECTORS[key]


def _run(name, two_s, two_M, B, dtype, irreps=None):
    torch = torch_cuda()
    F = ftlm()
    g = product_group(name)
    c = cluster(name)
    osec = _oracle_sector(name, two_s, two_M)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    worst = 0.0
    n_ir = len(oracle_group(name).irreps)
    for ir in (irreps if irreps is not None else range(n_ir)):
        ob = BlockBasis(osec, ir).with_hamiltonian(c.bonds)
        if ob.dim == 0:
            continue
        blk = F.ftlm_build_block(sec, ir)
        x = rand_block_vectors(ob.dim, B, seed=1000 * ir + B)
        y_ref = ob.hv(x)
        tdt = torch.float64 if dtype == F.F64 else torch.float32
        xd = torch.from_numpy(x).to("cuda", tdt).contiguous()
        yd = torch.full_like(xd, float("nan"))
        F.ftlm_hv(blk, dtype, B, xd, yd)
        F.ftlm_basis_check(blk)
        y = yd.double().cpu().numpy()
        scale = np.abs(y_ref).max() + 1e-300
        worst = max(worst, np.abs(y - y_ref).max() / scale)
    return worst


@pytest.mark.parametrize("name,two_s,two_M", CASES)
def test_hv_f64_matches_oracle(name, two_s, two_M):
    assert _run(name, two_s, two_M, 1, ftlm().F64) < 1e-13


@pytest.mark.parametrize("B", [2, 3, 8, 13, 32])
def test_hv_f64_batched(B):
    assert _run("icosahedron", 1, 2, B, ftlm().F64) < 1e-13
    assert _run("cuboctahedron", 3, 6, B, ftlm().F64, irreps=[0, 5, 9]) < 1e-13


@pytest.mark.parametrize("name,two_s,two_M", CASES[:6])
def test_hv_f32_matches_oracle(name, two_s, two_M):
    assert _run(name, two_s, two_M, 8, ftlm().F32) < 3e-6


def test_hv_symmetric_and_deterministic():
    """<u, H v> = <H u, v> (H is real symmetric in the block) and repeated launches are bitwise equal."""
    torch = torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")
    blk = F.ftlm_build_basis(g, 3, 0, 9)
    dim = F.ftlm_basis_info(blk)["dim"]
    u = torch.from_numpy(rand_block_vectors(dim, 1, 5)).cuda()
    v = torch.from_numpy(rand_block_vectors(dim, 1, 6)).cuda()
    hu, hv, hv2 = torch.empty_like(u), torch.empty_like(v), torch.empty_like(v)
    F.ftlm_hv(blk, F.F64, 1, u, hu)
    F.ftlm_hv(blk, F.F64, 1, v, hv)
    F.ftlm_hv(blk, F.F64, 1, v, hv2)
    torch.cuda.synchronize()
    a, b = float((u * hv).sum()), float((hu * v).sum())
    assert abs(a - b) < 1e-11 * (abs(a) + 1)
    assert torch.equal(hv, hv2)


def test_hv_rejects_bad_arguments():
    torch = torch_cuda()
    F = ftlm()
    blk = F.ftlm_build_basis(product_group("icosahedron"), 1, 0, 0)
    x = torch.zeros(F.ftlm_basis_info(blk)["dim"], 33, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FtlmError) as e:
        F.ftlm_hv(blk, F.F64, 33, x, x.clone())
    assert e.value.status == F.EINVAL
    with pytest.raises(F.FtlmError) as e:
        F.ftlm_hv(blk, F.F64, 0, x, x.clone())
    assert e.value.status == F.EINVAL
    with pytest.raises(F.FtlmError) as e:
        F.ftlm_build_basis(product_group("icosahedron"), 1, 1, 0)  # N s + M not an integer
    assert e.value.status == F.EINVAL


def _block_x_from_labels(labels_base_d, ng, off, B, seed, dtype):
    """Block vector whose rows depend only on (representative label, k, b): label-keyed inputs."""
    dmax = int(ng.max()) if len(ng) else 1
    vals = label_keyed_values(labels_base_d, dmax, B, seed)  # [n_reps, dmax, B]
    keep = np.arange(dmax)[None, :] < ng[:, None].astype(np.int64)
    X = vals[keep]
    assert X.shape[0] == int(off[-1])
    return X.astype(dtype)


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_hv_icosidodecahedron_m0_sampled_rows(dtype_name):
    """Full-size s=1/2 icosidodecahedron M=0 blocks, B = 8 as in the benchmark: sampled rows vs the oracle."""
    torch = torch_cuda()
    F = ftlm()
    name, two_s, two_M, B = "icosidodecahedron", 1, 0, 8
    og = oracle_group(name)
    c = cluster(name)
    g = product_group(name)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    rng = np.random.default_rng(11)
    # representatives to check, drawn from random sector states through the oracle
    sample = set()
    while len(sample) < 60:
        bits = rng.permutation(np.r_[np.ones(15, dtype=np.int64), np.zeros(15, dtype=np.int64)])
        lab = int(sum(int(v) << k for k, v in enumerate(bits)))
        sample.add(native.min_rep(og.n_sites, 2, og.perms, lab)[0])
    sample = sorted(sample)
    dtype, tdt, tol = ((F.F64, torch.float64, 1e-12) if dtype_name == "f64" else (F.F32, torch.float32, 2e-5))
    for ir in (0, 3, 6, 8):
        blk = F.ftlm_build_block(sec, ir)
        labels, _, ng, off = F.ftlm_basis_export(blk)
        X = _block_x_from_labels(labels, ng, off, B, 5, np.float64)
        xd = torch.from_numpy(X).to("cuda", tdt)
        yd = torch.empty_like(xd)
        F.ftlm_hv(blk, dtype, B, xd, yd)
        F.ftlm_basis_check(blk)
        Y = yd.double().cpu().numpy()
        rows = hv_rows_by_label(og, ir, c.bonds, 1.0, two_s, sample,
                                lambda lab, n: label_keyed_values([lab], n, B, 5)[0])
        pos = np.searchsorted(labels, np.array(sample, dtype=np.uint64))
        scale = np.abs(Y).max()
        for lab, p, yr in zip(sample, pos, rows):
            assert labels[p] == lab
            if yr is None:
                assert ng[p] == 0
                continue
            got = Y[int(off[p]):int(off[p]) + int(ng[p])]
            assert np.abs(got - yr).max() <= tol * scale


@pytest.mark.parametrize("name,two_s,two_M,B", [("icosahedron", 1, 0, 8), ("icosahedron", 1, 2, 1),
                                                ("icosahedron", 3, 4, 13), ("cuboctahedron", 2, 2, 8),
                                                ("square:4x4", 1, 0, 4)])
def test_hv_multi_matches_single_and_oracle(name, two_s, two_M, B):
    """One multi-block launch over all irreps = per-block H·v = oracle (FP64), and FP32 close."""
    torch = torch_cuda()
    F = ftlm()
    g = product_group(name)
    og = oracle_group(name)
    c = cluster(name)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    irreps = [i for i, ir in enumerate(og.irreps) if ir.dim <= 5][:16]
    mb = F.ftlm_build_multiblock(sec, irreps)
    dims = F.ftlm_multiblock_info(mb)["dims"]
    osec = _oracle_sector(name, two_s, two_M)
    for dtype, tdt, tol in ((F.F64, torch.float64, 1e-13), (F.F32, torch.float32, 3e-6)):
        xs, ys, refs = [], [], []
        for k, ir in enumerate(irreps):
            x = rand_block_vectors(max(dims[k], 1), B, seed=7 * k + B)[: dims[k]]
            xs.append(torch.from_numpy(np.ascontiguousarray(x)).to("cuda", tdt) if dims[k] else
                      torch.zeros(1, dtype=tdt, device="cuda"))
            ys.append(torch.full_like(xs[-1], float("nan")))
            refs.append(BlockBasis(osec, ir).with_hamiltonian(c.bonds).hv(x) if dims[k] else None)
        F.ftlm_hv_multi(mb, dtype, B, xs, ys)
        for k in range(len(irreps)):
            if dims[k] == 0:
                continue
            blk = F.ftlm_multiblock_block(mb, k)
            y1 = torch.empty_like(xs[k])
            F.ftlm_hv(blk, dtype, B, xs[k], y1)
            F.ftlm_basis_check(blk)
            scale = np.abs(refs[k]).max() + 1e-300
            assert np.abs(ys[k].double().cpu().numpy() - refs[k]).max() <= tol * scale
            assert np.abs(ys[k].double().cpu().numpy() - y1.double().cpu().numpy()).max() <= tol * scale


def test_lanczos_multi_matches_single():
    F = ftlm()
    g = product_group("icosahedron")
    sec = F.ftlm_build_sector(g, 3, 2)
    irreps = list(range(10))
    mb = F.ftlm_build_multiblock(sec, irreps)
    ids = [100 + k for k in irreps]
    a, b, st = F.ftlm_lanczos_multi(mb, F.F64, 5, 15, 9, ids)
    for k in irreps:
        blk = F.ftlm_multiblock_block(mb, k)
        a1, b1, s1 = F.ftlm_lanczos(blk, F.F64, 5, 15, 9, ids[k])
        assert np.array_equal(st[k], s1)
        assert np.allclose(a[k], a1, rtol=1e-10, atol=1e-10)
        assert np.allclose(b[k], b1, rtol=1e-10, atol=1e-10)
