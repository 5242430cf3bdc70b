"""Serving loop: jobs in a mix give the coefficients they give alone; admission respects the cap.

A job is one (M, Gamma) block with R chains (Section 2.2); in the mix it runs as
one part of a multi-sector packed Lanczos launch next to other jobs, alone it
runs through ftlm_lanczos.  Both are FP64 here, so the coefficients must agree
to rounding (1e-10 relative, the FP64 parity bar of the Lanczos tests).
"""
import numpy as np
import pytest

from gpu_common import ftlm, product_group, torch_cuda

pytestmark = pytest.mark.gpu


def _jobs(F):
    """A mix over three clusters, several M and irreps, R in {1, 4}, 16-30 steps."""
    rng = np.random.default_rng(11)
    out = []
    for name, two_s, Ms in (("icosahedron", 1, (0, 2, 4, 6)), ("cuboctahedron", 1, (0, 2, 4)),
                            ("square:4x4", 1, (0, 2, 4))):
        g = product_group(name)
        dims = F.ftlm_group_info(g)["dims"]
        for two_M in Ms:
            sec = F.ftlm_build_sector(g, two_s, two_M)
            for ir in range(len(dims)):
                if int(dims[ir]) > 5:
                    continue
                if F.ftlm_basis_info(F.ftlm_build_block(sec, ir))["dim"] == 0:
                    continue
                if rng.random() < 0.45:
                    out.append(dict(g=g, two_s=two_s, two_M=two_M, irrep=ir, R=int(rng.choice([1, 4])),
                                    n_steps=int(rng.integers(16, 31)), block_id=64 * two_M + ir))
    return out


def test_jobs_in_the_mix_match_each_job_alone():
    torch_cuda()
    F = ftlm()
    jobs = _jobs(F)
    assert len(jobs) >= 20
    srv = F.Server(cap_bytes=8 << 30, n_workers=3, max_parts=16)
    try:
        ids = [srv.submit(j["g"], j["two_s"], j["two_M"], j["irrep"], j["R"], j["n_steps"], 7, j["block_id"],
                          F.GAUSS, F.F64) for j in jobs]
        res = [srv.wait(i, 300.0) for i in ids]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["completed"] == len(jobs) and stats["failed"] == 0
    assert stats["parts"] == len(jobs) and 1 <= stats["waves"] <= len(jobs)
    assert stats["sector_hits"] > 0  # jobs on the same sector reused its tables
    for j, (info, a, b, st) in zip(jobs, res):
        blk = F.ftlm_build_basis(j["g"], j["two_s"], j["two_M"], j["irrep"])
        a1, b1, s1 = F.ftlm_lanczos(blk, F.F64, j["R"], j["n_steps"], 7, j["block_id"], F.GAUSS)
        assert info["status"] == F.OK and info["dim"] == F.ftlm_basis_info(blk)["dim"]
        assert info["t_submit"] <= info["t_admit"] <= info["t_start"] <= info["t_done"]
        assert np.array_equal(st, s1)
        for r in range(j["R"]):
            k = s1[r]
            scale = np.abs(a1[r, :k]).max() + 1.0
            assert np.abs(a[r, :k] - a1[r, :k]).max() <= 1e-10 * scale
            assert np.abs(b[r, :k] - b1[r, :k]).max() <= 1e-10 * scale
            assert np.all(a[r, k:] == 0) and np.all(b[r, k:] == 0)


def test_admission_cap_is_respected_and_tables_are_evicted():
    torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")
    dims = F.ftlm_group_info(g)["dims"]
    cap = 48 << 20  # a few jobs at a time: forces waiting, eviction and reuse
    srv = F.Server(cap_bytes=cap, n_workers=2, max_parts=4)
    try:
        ids = []
        for two_M in (0, 2, 4, 6, 8):
            for ir in range(len(dims)):
                ids.append(srv.submit(g, 1, two_M, ir, 4, 20, 3, 64 * two_M + ir, F.RADEMACHER, F.F32))
        done = 0
        for i in ids:
            try:
                srv.wait(i, 300.0)
                done += 1
            except F.FtlmError as e:  # empty blocks have nothing to run
                assert e.status in (F.EINVAL, F.EUNSUPPORTED)
        stats = srv.stats()
    finally:
        srv.close()
    assert done > 0
    assert stats["peak_charged"] <= cap
    assert stats["charged"] <= cap


def test_job_too_large_for_the_cap_fails_and_others_complete():
    torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")
    srv = F.Server(cap_bytes=12 << 20, n_workers=1, max_parts=4)
    try:
        small = srv.submit(g, 1, 4, 0, 1, 10, 1, 0)
        big = srv.submit(g, 3, 0, 9, 32, 40, 1, 1)  # s = 3/2, M = 0: tables and vectors far above 12 MB
        after = srv.submit(g, 1, 6, 0, 1, 10, 1, 2)
        srv.wait(small, 120.0)
        with pytest.raises(F.FtlmError) as e:
            srv.wait(big, 120.0)
        assert e.value.status == F.ENOMEM
        srv.wait(after, 120.0)
    finally:
        srv.close()


def test_submit_rejects_bad_jobs():
    torch_cuda()
    F = ftlm()
    g = product_group("icosahedron")
    srv = F.Server(cap_bytes=1 << 30)
    try:
        for kw in (dict(R=0), dict(R=33), dict(n_steps=0), dict(irrep=10), dict(two_M=1)):
            args = dict(two_s=1, two_M=0, irrep=0, R=2, n_steps=10)
            args.update(kw)
            with pytest.raises(F.FtlmError) as e:
                srv.submit(g, args["two_s"], args["two_M"], args["irrep"], args["R"], args["n_steps"], 1, 0)
            assert e.value.status == F.EINVAL
    finally:
        srv.close()


def test_real_form_and_wide_irrep_jobs():
    """Jobs on irreps of complex type (C_12, AGL(1,11)), quaternionic type (Q_8) and of dimension 6 and 10
    (S_5 on the Petersen graph, AGL(1,11)): in the mix they give the coefficients they give alone, and their
    info carries the irrep's weight."""
    torch_cuda()
    F = ftlm()
    jobs = []
    for name, two_s, Ms in (("chain:12", 1, (0, 2)), ("complete:11", 2, (0,)), ("petersen", 2, (0, 2)),
                            ("q8", 3, (2,))):
        g = product_group(name)
        info = F.ftlm_group_info(g)
        for two_M in Ms:
            sec = F.ftlm_build_sector(g, two_s, two_M)
            for ir in range(len(info["dims"])):
                if info["fs"][ir] == 1 and info["dims"][ir] < 6:
                    continue  # complex-type real forms and d = 6 only
                if F.ftlm_basis_info(F.ftlm_build_block(sec, ir))["dim"] < 64:
                    continue  # Krylov spaces of real-form blocks exhaust at dim / kappa: keep 12 steps below that
                jobs.append(dict(g=g, two_s=two_s, two_M=two_M, irrep=ir, R=2, n_steps=12,
                                 block_id=64 * two_M + ir, weight=int(info["weights"][ir])))
    assert len(jobs) >= 6
    srv = F.Server(cap_bytes=4 << 30, n_workers=2, max_parts=8)
    try:
        ids = [srv.submit(j["g"], j["two_s"], j["two_M"], j["irrep"], j["R"], j["n_steps"], 5, j["block_id"],
                          F.GAUSS, F.F64) for j in jobs]
        res = [srv.wait(i, 300.0) for i in ids]
    finally:
        srv.close()
    for j, (info, a, b, st) in zip(jobs, res):
        blk = F.ftlm_build_basis(j["g"], j["two_s"], j["two_M"], j["irrep"])
        a1, b1, s1 = F.ftlm_lanczos(blk, F.F64, j["R"], j["n_steps"], 5, j["block_id"], F.GAUSS)
        assert info["status"] == F.OK and info["d_gamma"] == j["weight"]
        assert np.array_equal(st, s1)
        for r in range(j["R"]):
            k = s1[r]
            scale = np.abs(a1[r, :k]).max() + 1.0
            assert np.abs(a[r, :k] - a1[r, :k]).max() <= 1e-10 * scale
            assert np.abs(b[r, :k] - b1[r, :k]).max() <= 1e-10 * scale
