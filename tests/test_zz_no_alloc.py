"""ftlm_thermo_noalloc: the thermal sums for callers that cannot allocate device memory.

Some callers run inside a process whose device memory is fully reserved by
another allocator or pool, or must avoid the device-wide synchronisation that
cudaMalloc/cudaFree can cause; the no-allocation entry point serves them from
a fixed scratch array.  This file is collected last.  It checks the entry
point against ftlm_thermo on two calls in a row (the scratch keeps the previous
call's contents) and that oversized inputs are rejected.
"""
import numpy as np
import pytest

from gpu_common import ftlm, product_group, torch_cuda

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


def test_noalloc_thermo_rejects_oversize():
    torch = torch_cuda()
    F = ftlm()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    mi = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(F.FtlmError) as e:
        F.ftlm_thermo_noalloc(1 << 14, 64, mi, x, x, x, x, 1, x, 1.0, x, x)  # 2^20 entries > 2^19
    assert e.value.status == F.EINVAL
    assert "fixed scratch" in F.ftlm_last_error()
    with pytest.raises(F.FtlmError) as e:
        F.ftlm_thermo_noalloc(4, 600, mi, x, x, x, x, 1, x, 1.0, x, x)
    assert e.value.status == F.EINVAL
