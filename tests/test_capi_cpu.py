"""C-ABI library checks that need no GPU: symbols, host group module vs oracle, error paths."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.group import Group
from workloads import cluster

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ftlm():
    from paper_2607_17429_gb300 import build

    build.build()
    from paper_2607_17429_gb300 import ftlm as F

    return F


def test_library_exports_every_declared_symbol(ftlm):
    with open(os.path.join(ROOT, "include", "ftlm.h")) as f:
        text = f.read()
    declared = set(re.findall(r"^\s*(?:ftlm_status|void|const char \*)\s*(ftlm_\w+)\s*\(", text, re.M))
    assert len(declared) >= 20
    lib = ctypes.CDLL(ftlm.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(ftlm.EXPORTED)


@pytest.mark.parametrize("name", ["dimer", "ring:5", "tetrahedron", "cuboctahedron", "icosahedron", "dodecahedron",
                                  "icosidodecahedron", "square:4x4", "square:4x6"])
def test_builtin_groups_match_oracle(ftlm, name):
    g = ftlm.ftlm_group_builtin(name)
    info = ftlm.ftlm_group_info(g)
    _, perms = ftlm.ftlm_group_irrep(g)
    bonds, J = ftlm.ftlm_group_bonds(g)
    c = cluster(name)
    og = Group(c.gens, c.bonds)
    assert np.array_equal(perms, og.perms)
    assert np.array_equal(bonds, c.bonds) and J == 1.0
    assert list(info["dims"]) == [ir.dim for ir in og.irreps]
    assert np.abs(info["chars"] - og.char_table).max() < 1e-10
    for i, ir in enumerate(og.irreps):
        rho, _ = ftlm.ftlm_group_irrep(g, i)
        # homomorphism and orthogonality of the library's own matrices
        assert np.abs(np.einsum("gab,hbc->ghac", rho, rho) - rho[og.mult]).max() < 1e-10
        assert np.abs(np.einsum("gab,gcb->gac", rho, rho) - np.eye(ir.dim)).max() < 1e-10


@pytest.mark.parametrize("name", ["square:4x4:t", "chain:8", "tetrahedron:t", "complete:7", "complete:11",
                                  "petersen", "q8"])
def test_real_forms_match_oracle(ftlm, name):
    """Irreps of complex and quaternionic type in real form (the library's reading of Section 3's
    complex path) and dimensions above 5: the library's own irreps, computed from generators,
    agree with the oracle's in dimension, type, weight and character, in the same canonical order."""
    c = cluster(name)
    g = ftlm.ftlm_group_init(c.gens, c.bonds)
    og = Group(c.gens, c.bonds)
    info = ftlm.ftlm_group_info(g)
    assert list(info["dims"]) == [ir.dim for ir in og.irreps]
    assert list(info["fs"]) == [ir.fs for ir in og.irreps]
    assert list(info["weights"]) == [ir.weight for ir in og.irreps]
    assert np.abs(info["chars"] - og.char_table).max() < 1e-10
    for i, ir in enumerate(og.irreps):
        rho, _ = ftlm.ftlm_group_irrep(g, i)
        assert np.abs(np.einsum("gab,hbc->ghac", rho, rho) - rho[og.mult]).max() < 1e-10
        assert np.abs(np.einsum("gab,gcb->gac", rho, rho) - np.eye(ir.dim)).max() < 1e-10
    if name == "square:4x4:t":  # k in {0, pi}^2 real; 12 complex momenta in 6 pairs
        assert list(info["fs"]).count(1) == 4 and list(info["fs"]).count(0) == 6


def test_group_init_from_generators(ftlm):
    c = cluster("cuboctahedron")
    g = ftlm.ftlm_group_init(c.gens, c.bonds, J=0.5)
    assert ftlm.ftlm_group_info(g)["order"] == 48
    assert ftlm.ftlm_group_bonds(g)[1] == 0.5


def test_set_irreps_tabulated(ftlm):
    c = cluster("icosahedron")
    og = Group(c.gens, c.bonds)
    g = ftlm.ftlm_group_init(c.gens, c.bonds)
    # hand the oracle's matrices over in a scrambled order; the library re-sorts canonically
    rhos = [ir.rho for ir in og.irreps][::-1]
    ftlm.ftlm_group_set_irreps(g, rhos)
    for i, ir in enumerate(og.irreps):
        rho, _ = ftlm.ftlm_group_irrep(g, i)
        assert np.array_equal(rho, ir.rho)


@pytest.mark.parametrize("name", ["q8", "complete:7", "chain:6"])
def test_set_irreps_real_forms(ftlm, name):
    """Tabulated real forms: the type follows from <chi, chi> = 1, 2, 4."""
    c = cluster(name)
    og = Group(c.gens, c.bonds)
    g = ftlm.ftlm_group_init(c.gens, c.bonds)
    ftlm.ftlm_group_set_irreps(g, [ir.rho for ir in og.irreps][::-1])
    info = ftlm.ftlm_group_info(g)
    assert list(info["fs"]) == [ir.fs for ir in og.irreps]
    assert list(info["weights"]) == [ir.weight for ir in og.irreps]
    # a complex-type real form with one row dropped is no representation: rejected, group unchanged
    bad = [ir.rho if ir.fs == 1 else ir.rho[:, :1, :1] for ir in og.irreps]
    with pytest.raises(ftlm.FtlmError) as e:
        ftlm.ftlm_group_set_irreps(g, bad)
    assert e.value.status == ftlm.EIRREP
    assert list(ftlm.ftlm_group_info(g)["fs"]) == [ir.fs for ir in og.irreps]


def test_error_paths(ftlm):
    c = cluster("icosahedron")
    with pytest.raises(ftlm.FtlmError) as e:
        ftlm.ftlm_group_init(np.array([[0, 0, 1]]), np.array([[0, 1]]))
    assert e.value.status == ftlm.ENOTGROUP
    with pytest.raises(ftlm.FtlmError) as e:
        ftlm.ftlm_group_init(c.gens, c.bonds[:-1])
    assert e.value.status == ftlm.EBONDS
    with pytest.raises(ftlm.FtlmError) as e:
        ftlm.ftlm_group_builtin("kagome:36")
    assert e.value.status == ftlm.EINVAL
    g = ftlm.ftlm_group_init(c.gens, c.bonds)
    og = Group(c.gens, c.bonds)
    bad = [ir.rho.copy() for ir in og.irreps]
    bad[3][5] *= -1.0  # breaks the homomorphism
    with pytest.raises(ftlm.FtlmError) as e:
        ftlm.ftlm_group_set_irreps(g, bad)
    assert e.value.status == ftlm.EIRREP
    with pytest.raises(ftlm.FtlmError) as e:
        ftlm.ftlm_group_set_irreps(g, [ir.rho for ir in og.irreps][:-1])  # incomplete
    assert e.value.status == ftlm.EIRREP
    assert "sum of d^2" in ftlm.ftlm_last_error()


def test_binding_checks_device_arrays(ftlm):
    """The binding passes a tensor's address only for a contiguous CUDA tensor of the right element type and
    size; raw integer addresses pass unchecked (the C-ABI's contract)."""
    torch = pytest.importorskip("torch")
    x = torch.zeros(16, dtype=torch.float64)
    with pytest.raises(ValueError, match="not on a CUDA device"):
        ftlm._dev(x, "float64", 16, "x")
    assert ftlm._dev(None) is None and ftlm._dev(12345) == 12345
    with pytest.raises(TypeError, match="CUDA tensor or a device address"):
        ftlm._dev(np.zeros(4), "float64", 4, "x")

    class FakeCuda:  # stands in for a CUDA tensor on a machine without a GPU
        def __init__(self, dtype, n, contiguous=True):
            self.is_cuda, self.dtype, self.n, self.c = True, dtype, n, contiguous

        def is_contiguous(self):
            return self.c

        def numel(self):
            return self.n

        def data_ptr(self):
            return 4096

    assert ftlm._dev(FakeCuda(torch.float32, 8), "float32", 8, "x") == 4096
    with pytest.raises(TypeError, match="element type"):
        ftlm._dev(FakeCuda(torch.float64, 8), "float32", 8, "x")
    with pytest.raises(ValueError, match="at least 9"):
        ftlm._dev(FakeCuda(torch.float32, 8), "float32", 9, "x")
    with pytest.raises(ValueError, match="not contiguous"):
        ftlm._dev(FakeCuda(torch.float32, 8, False), "float32", 8, "x")
    assert ftlm._vt(ftlm.F32) == "float32" and ftlm._vt(ftlm.F64) == "float64"
