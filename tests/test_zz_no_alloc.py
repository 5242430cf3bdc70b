"""ftlm_thermo_noalloc: the thermal sums for callers that cannot allocate device memory.

Some callers run inside a process whose device memory is fully reserved by
another allocator or pool, or must avoid the device-wide synchronisation that
cudaMalloc/cudaFree can cause; the no-allocation entry point serves them from
a fixed scratch array.  This file is collected last.  It checks the entry
point against ftlm_thermo on two calls in a row (the scratch keeps the previous
call's contents), a third smaller call against the oracle's thermal sums
(Eqs. 5-7, 14), that a call after the warm-up form leaves the device's free
memory unchanged, that the error word of a failed call is cleared by the next
one, and that oversized inputs are rejected.
"""
import numpy as np
import pytest

from gpu_common import ftlm, product_group, torch_cuda
from oracle.lanczos import thermo as oracle_thermo

pytestmark = pytest.mark.gpu


def _blocks(F, name, two_s, Ms, R, steps, seed):
    g = product_group(name)
    dims = F.ftlm_group_info(g)["dims"]
    out = []
    for two_M in Ms:
        sec = F.ftlm_build_sector(g, two_s, two_M)
        for ir in range(len(dims)):
            blk = F.ftlm_build_block(sec, ir)
            dim = F.ftlm_basis_info(blk)["dim"]
            if dim == 0:
                continue
            a, b, st = F.ftlm_lanczos(blk, F.F64, R, steps, seed, 64 * two_M + ir)
            out.append(dict(two_M=two_M, d_gamma=int(dims[ir]), dim=dim, alpha=a, beta=b, steps=st))
    return out


def _device_inputs(torch, blocks, ld):
    alpha, beta, m, weight, msq = [], [], [], [], []
    for bl in blocks:
        R = bl["alpha"].shape[0]
        mult = 2.0 if bl["two_M"] > 0 else 1.0
        for r in range(R):
            a = np.zeros(ld)
            b = np.zeros(ld)
            k = bl["alpha"].shape[1]
            a[:k], b[:k] = bl["alpha"][r], bl["beta"][r]
            alpha.append(a)
            beta.append(b)
            m.append(int(bl["steps"][r]))
            weight.append(mult * bl["d_gamma"] * bl["dim"] / R)
            msq.append((bl["two_M"] / 2.0) ** 2)
    dev = dict(alpha=torch.tensor(np.array(alpha), device="cuda"), beta=torch.tensor(np.array(beta), device="cuda"),
               m=torch.tensor(np.array(m, dtype=np.int32), device="cuda"),
               weight=torch.tensor(np.array(weight), device="cuda"), msq=torch.tensor(np.array(msq), device="cuda"))
    return dev, len(m)


def _noalloc(F, torch, blocks, ld, T, g):
    dev, n_chains = _device_inputs(torch, blocks, ld)
    Td = torch.tensor(T, device="cuda")
    out = torch.full((4, len(T)), float("nan"), dtype=torch.float64, device="cuda")
    E0 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    F.ftlm_thermo_noalloc(n_chains, ld, dev["m"], dev["alpha"], dev["beta"], dev["weight"], dev["msq"], len(T), Td,
                          g, out, E0)
    o = out.cpu().numpy()
    return o[0], o[1], o[2], o[3], float(E0.item())


def test_noalloc_thermo_matches_ftlm_thermo_twice():
    torch = torch_cuda()
    F = ftlm()
    T1 = 0.02 * 5000.0 ** (np.arange(200) / 199.0)
    T2 = np.geomspace(0.05, 20.0, 37)
    calls = [(_blocks(F, "icosahedron", 1, range(0, 13, 2), 4, 30, 0), 30, T1, 1.0),
             (_blocks(F, "cuboctahedron", 2, range(0, 25, 2), 3, 40, 5), 48, T2, 2.0)]
    for blocks, ld, T, g in calls:  # two calls in a row on the shared scratch
        ref = F.ftlm_thermo(blocks, T, g)
        got = _noalloc(F, torch, blocks, ld, T, g)
        assert abs(got[4] - ref[4]) <= 1e-12 * abs(ref[4])
        for a, b in zip(got[:4], ref[:4]):
            assert np.all(np.isfinite(a))
            assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())


def test_noalloc_third_call_matches_oracle_and_allocates_nothing():
    torch = torch_cuda()
    F = ftlm()
    F.ftlm_thermo_noalloc(0, 0, None, None, None, None, None, 0, None, 1.0, None, None)  # warm-up form
    blocks = _blocks(F, "icosahedron", 1, range(0, 13, 4), 2, 12, 9)
    T = np.geomspace(0.1, 10.0, 11)
    dev, n_chains = _device_inputs(torch, blocks, 12)
    Td = torch.tensor(T, device="cuda")
    out = torch.full((4, len(T)), float("nan"), dtype=torch.float64, device="cuda")
    E0 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    F.ftlm_thermo_noalloc(n_chains, 12, dev["m"], dev["alpha"], dev["beta"], dev["weight"], dev["msq"], len(T), Td,
                          1.0, out, E0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref = oracle_thermo([dict(two_M=bl["two_M"], d_gamma=bl["d_gamma"], dim=bl["dim"], R=bl["alpha"].shape[0],
                              alpha=[a[:k] for a, k in zip(bl["alpha"], bl["steps"])],
                              beta=[b[:k] for b, k in zip(bl["beta"], bl["steps"])]) for bl in blocks], T, 1.0)
    o = out.cpu().numpy()
    assert abs(float(E0.item()) - ref[4]) <= 1e-10 * abs(ref[4])
    for a, b in zip(o, ref[:4]):
        assert np.abs(a - b).max() <= 1e-10 * max(1.0, np.abs(b).max())


def test_noalloc_error_word_is_cleared_by_the_next_call():
    torch = torch_cuda()
    F = ftlm()
    blocks = _blocks(F, "icosahedron", 1, [0, 2], 2, 10, 3)
    dev, n_chains = _device_inputs(torch, blocks, 10)
    T = np.array([0.5, 1.0, 2.0])
    Td = torch.tensor(T, device="cuda")
    out = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    E0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    bad = dev["m"].clone()
    bad[0] = 11  # more steps than the leading dimension: the Ritz kernel flags it and reads nothing
    with pytest.raises(F.FtlmError) as e:
        F.ftlm_thermo_noalloc(n_chains, 10, bad, dev["alpha"], dev["beta"], dev["weight"], dev["msq"], 3, Td, 1.0,
                              out, E0)
    assert e.value.status == F.EINTERNAL
    F.ftlm_thermo_noalloc(n_chains, 10, dev["m"], dev["alpha"], dev["beta"], dev["weight"], dev["msq"], 3, Td, 1.0,
                          out, E0)
    ref = F.ftlm_thermo(blocks, T, 1.0)
    assert abs(float(E0.item()) - ref[4]) <= 1e-12 * abs(ref[4])


def test_noalloc_thermo_rejects_oversize():
    torch = torch_cuda()
    F = ftlm()
    xt = torch.zeros(8, dtype=torch.float64, device="cuda")
    mt = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError, match="at least"):  # the binding checks tensor sizes first
        F.ftlm_thermo_noalloc(1 << 14, 64, mt, xt, xt, xt, xt, 1, xt, 1.0, xt, xt)
    # raw addresses pass the binding unchecked: the library rejects the sizes before any GPU work
    x, mi = xt.data_ptr(), mt.data_ptr()
    with pytest.raises(F.FtlmError) as e:
        F.ftlm_thermo_noalloc(1 << 14, 64, mi, x, x, x, x, 1, x, 1.0, x, x)  # 2^20 entries > 2^19
    assert e.value.status == F.EINVAL
    assert "fixed scratch" in F.ftlm_last_error()
    with pytest.raises(F.FtlmError) as e:
        F.ftlm_thermo_noalloc(4, 600, mi, x, x, x, x, 1, x, 1.0, x, x)
    assert e.value.status == F.EINVAL
