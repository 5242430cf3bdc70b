"""GPU basis tables vs the oracle: bit-exact representatives, stabilizers, n_Gamma and offsets."""
import numpy as np
import pytest

from gpu_common import ftlm, product_group
from helpers import masks_from_words, oracle_group, pack_labels, unpack_label
from oracle import native
from oracle.basis import BlockBasis, SectorBasis
from oracle.sector import block_dims, fixed_count, sector_dim

pytestmark = pytest.mark.gpu

CASES = [("icosahedron", 1, 0), ("icosahedron", 1, 6), ("icosahedron", 1, 12), ("icosahedron", 3, 0),
         ("cuboctahedron", 1, 0), ("cuboctahedron", 2, 2), ("tetrahedron", 5, 2), ("ring:7", 1, 1),
         ("square:4x4", 1, 0), ("square:4x6", 1, 4), ("dodecahedron", 1, 0), ("dimer", 1, 0),
         ("ring:6", 5, 0), ("cuboctahedron", 3, 12), ("icosahedron", 1, -4),
         ("cuboctahedron", 4, 32)]  # s = 2: 36-bit labels, most representatives above 2^32


@pytest.mark.parametrize("name,two_s,two_M", CASES)
def test_basis_bit_exact(name, two_s, two_M):
    F = ftlm()
    g = product_group(name)
    og = oracle_group(name)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    info = F.ftlm_sector_info(sec)
    osec = SectorBasis(og, two_s, two_M)
    assert info["sector_dim"] == sector_dim(og.n_sites, two_s, two_M)
    assert info["n_reps"] == osec.n_reps
    labels, masks = F.ftlm_sector_export(sec)
    assert np.array_equal(labels, pack_labels(osec.reps, og.n_sites, two_s))
    assert np.array_equal(masks, masks_from_words(osec.stab, og.order))
    for ir in range(len(og.irreps)):
        blk = F.ftlm_build_block(sec, ir)
        ob = BlockBasis(osec, ir)
        _, _, ng, off = F.ftlm_basis_export(blk)
        assert np.array_equal(ng.astype(np.int64), ob.n.astype(np.int64))
        assert np.array_equal(off.astype(np.int64), ob.off)
        assert F.ftlm_basis_info(blk)["dim"] == ob.dim


def test_icosidodecahedron_m0_sector_counts():
    """Full-size sector of the s=1/2 icosidodecahedron (M=0): counts and sampled representatives."""
    F = ftlm()
    name, two_s, two_M = "icosidodecahedron", 1, 0
    g = product_group(name)
    og = oracle_group(name)
    sec = F.ftlm_build_sector(g, two_s, two_M)
    info = F.ftlm_sector_info(sec)
    assert info["sector_dim"] == 155117520
    burnside = sum(fixed_count(p, two_s, two_M) for p in og.perms) // og.order
    assert info["n_reps"] == burnside
    labels, masks = F.ftlm_sector_export(sec)
    assert np.all(np.diff(labels.astype(np.int64)) > 0)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(labels), 300, replace=False):
        lab = unpack_label(int(labels[i]), og.n_sites, two_s)
        rep, gs = native.min_rep(og.n_sites, 2, og.perms, lab)
        assert rep == lab
    dims = block_dims(og, two_s, two_M)
    for ir in range(len(og.irreps)):
        blk = F.ftlm_build_block(sec, ir)
        assert F.ftlm_basis_info(blk)["dim"] == dims[ir]
