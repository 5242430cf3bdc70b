#!/usr/bin/env python
"""Benchmark: symmetry-adapted FTLM of the s=1/2 icosidodecahedron, M = 0, all 10 I_h irreps.

One step = one full pass of the hot path over the workload: enumerate the M = 0
sector on the GPU (1.55e8 states -> orbit representatives, stabilizers, lookup
index), build the 10 irrep blocks and their packed set, run R = 8 Lanczos
chains of 60 steps on every block (each step one packed H·v launch over all ten
blocks with B = 8 right-hand sides, FP32 vectors, FP64 alpha/beta), Ritz pairs
and thermal sums on 200 temperatures.

value    = state-applications per second: sum over blocks of dim * chains * steps
           done, divided by the device time of the steps (group tables resident).
e2e      = the same metric through the public C-ABI calls from host buffers
           (generators and bonds uploaded, alpha/beta and thermal curves read back).
roofline = the packed H·v kernel (the dominant launch), timed with CUDA events
           recorded inside the Lanczos graph; algorithmic bytes per launch as in
           the kernel's roofline definition (gathers of every flipped state's
           segment, the representative's own rows in and out, the lookups).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "icosidodecahedron s=1/2 M=0, I_h all 10 irreps, R=8 Gaussian (seed 1), 60 Lanczos steps"
METRIC = "sym-adapted H·v Gstates/s (FTLM step: enumeration + 10 irrep blocks x 8 chains x 60 Lanczos steps + thermo)"
CLUSTER, TWO_S, TWO_M, R, N_STEPS, SEED = "icosidodecahedron", 1, 0, 8, 60, 1
T_GRID = 0.02 * 5000.0 ** (np.arange(200) / 199.0)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x):
    """Largest value of x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(states_per_rank, ms_all, world):
    """Whole-job Gstates/s of `world` replicas that each processed `states_per_rank` in at most ms_all ms."""
    return states_per_rank * world / (ms_all / 1e3) / 1e9


def run_ours(args, rank, world):
    import torch

    from paper_2607_17429_gb300 import build as pb

    pb.build()
    from paper_2607_17429_gb300 import ftlm as F
    from workloads import cluster

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    dtype = F.F32 if args.dtype == "f32" else F.F64
    c = cluster(CLUSTER)
    gens, bonds = np.ascontiguousarray(c.gens), np.ascontiguousarray(c.bonds)
    group = F.ftlm_group_init(gens, bonds)  # resident inputs for the device-timed value
    dims_g = F.ftlm_group_info(group)["dims"]
    n_ir = len(dims_g)
    ids = [64 * TWO_M + ir for ir in range(n_ir)]

    def step_multi(grp, dt, flips=None):
        """Batched form: all 10 irrep blocks through one packed H·v launch per Lanczos step; with the entry
        table, the sector's flips are searched once per step and every H·v reads them."""
        sec = F.ftlm_build_sector(grp, TWO_S, TWO_M, stream)
        if (flips or args.flips) == "table":
            F.ftlm_sector_build_entries(sec, stream)
        mb = F.ftlm_build_multiblock(sec, list(range(n_ir)), stream)
        dims = F.ftlm_multiblock_info(mb)["dims"]
        a, b, st = F.ftlm_lanczos_multi(mb, dt, R, N_STEPS, SEED, ids, F.GAUSS, stream)
        blocks = [dict(two_M=TWO_M, d_gamma=int(dims_g[k]), dim=dims[k], alpha=a[k], beta=b[k], steps=st[k])
                  for k in range(n_ir)]
        states = sum(dims[k] * int(st[k].sum()) for k in range(n_ir))
        return states, F.ftlm_thermo(blocks, T_GRID, 1.0, stream)

    def step_single(grp, dt):
        """Plain form: one block at a time, one H·v launch per block and Lanczos step."""
        sec = F.ftlm_build_sector(grp, TWO_S, TWO_M, stream)
        blocks, states = [], 0
        for ir in range(n_ir):
            blk = F.ftlm_build_block(sec, ir, stream)
            dim = F.ftlm_basis_info(blk)["dim"]
            a, b, st = F.ftlm_lanczos(blk, dt, R, N_STEPS, SEED, ids[ir], F.GAUSS, stream)
            blocks.append(dict(two_M=TWO_M, d_gamma=int(dims_g[ir]), dim=dim, alpha=a, beta=b, steps=st))
            states += dim * int(st.sum())
        return states, F.ftlm_thermo(blocks, T_GRID, 1.0, stream)

    step = step_multi

    def timed(dt, K, W, fn=None):
        fn = fn or step
        for _ in range(W):
            fn(group, dt)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        F.ftlm_profile_reset()
        F.ftlm_profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        states = 0
        out = None
        for _ in range(K):
            s, out = fn(group, dt)
            states += s
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        F.ftlm_profile_enable(False)
        prof = F.ftlm_profile_get()
        ms = e0.elapsed_time(e1)
        return ms, states, prof, out

    with Clocks(dev) as clk:
        ms, states, prof, out = timed(dtype, args.steps, args.warmup)
    ms_all = max_over_ranks(ms)  # the slowest replica's time
    value = replica_value(states, ms_all, world)  # replicas: every rank runs the same workload
    res = {"ms": ms, "states": states, "prof": prof, "out": out, "clocks": clk.summary(), "value": value,
           "ms_all": ms_all}
    # algorithmic counts of one packed H·v launch (for the roofline)
    sec = F.ftlm_build_sector(group, TWO_S, TWO_M, stream)
    labels, _ = F.ftlm_sector_export(sec)
    mb = F.ftlm_build_multiblock(sec, list(range(n_ir)), stream)
    res.update(flips=_flip_count(labels, bonds), n_reps=len(labels), W=int(sum(int(d) for d in dims_g)),
               rows=F.ftlm_multiblock_packed_rows(mb), dims=F.ftlm_multiblock_info(mb)["dims"])
    del mb, sec

    # FP64 companions: the plain one-block-at-a-time form and the batched form (mixed vs FP64 error)
    fp64 = None
    if not args.skip_fp64 and dtype == F.F32:
        fp64 = {}
        for name, fn in (("plain_single_block", step_single), ("batched", step_multi)):
            ms64, st64, prof64, out64 = timed(F.F64, 1, 1, fn)
            fp64[name] = {"value": st64 / (ms64 / 1e3) / 1e9, "ms_per_step": ms64,
                          "blocks_per_hour": n_ir / (ms64 / 1e3) * 3600.0,
                          "hv_ms_per_launch": prof64["hv_ms"] / max(1, prof64["hv_launches"]), "E0": out64[4]}
        ref = out64  # FP64 batched
        sel = T_GRID >= 0.05
        fp64["mixed_vs_fp64"] = {
            "dE0_rel": abs(out[4] - ref[4]) / abs(ref[4]),
            "max_dC_over_Cmax": float(np.abs(out[2] - ref[2])[sel].max() / ref[2].max()),
            "max_dlnZ_rel": float(np.abs((out[0] - ref[0]) / ref[0]).max()),
            "chi": "identically 0 in an M = 0-only run (chi needs M != 0 sectors)"}
        fp64["batched_mixed_over_plain_fp64_blocks_per_hour"] = (
            (n_ir * args.steps / (ms / 1e3)) / (n_ir / (fp64["plain_single_block"]["ms_per_step"] / 1e3)))
        # FP16 storage (FP32 arithmetic, FP64 reductions), batched form, same seed
        ms16, st16, prof16, out16 = timed(F.F16, 1, 1, step_multi)
        res["fp16_storage"] = {
            "value": st16 / (ms16 / 1e3) / 1e9, "unit": "Gstates/s", "ms_per_step": ms16,
            "hv_ms_per_launch": prof16["hv_ms"] / max(1, prof16["hv_launches"]), "E0": out16[4],
            "vs_fp64": {"dE0_rel": abs(out16[4] - ref[4]) / abs(ref[4]),
                        "max_dC_over_Cmax": float(np.abs(out16[2] - ref[2])[sel].max() / ref[2].max()),
                        "max_dlnZ_rel": float(np.abs((out16[0] - ref[0]) / ref[0]).max())}}

    # e2e: public API from host buffers, wall clock, copies inside
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_states = 0
    for _ in range(args.steps):
        g2 = F.ftlm_group_init(gens, bonds)
        s2, out2 = step(g2, dtype)
        e2e_states += s2
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    h2d = gens.nbytes + bonds.nbytes + T_GRID.nbytes
    d2h = n_ir * R * N_STEPS * 8 * 2 + n_ir * R * 4 + 4 * len(T_GRID) * 8 + 8
    res["e2e"] = {"value": e2e_states / t_e2e / 1e9, "unit": "Gstates/s", "h2d_bytes_per_step": int(h2d),
                  "d2h_bytes_per_step": int(d2h)}
    res["fp64"] = fp64
    # the other flip path on the same workload (entry table vs on-the-fly search)
    other = "search" if args.flips == "table" else "table"
    ms_o, st_o, prof_o, out_o = timed(dtype, 1, 1, lambda grp, dt: step_multi(grp, dt, other))
    res["other_flip_path"] = {"flips": other, "value": st_o / (ms_o / 1e3) / 1e9, "unit": "Gstates/s",
                              "ms_per_step": ms_o, "hv_ms_per_launch": prof_o["hv_ms"] / max(1, prof_o["hv_launches"]),
                              "dE0_vs_headline": abs(out_o[4] - out[4])}
    # measured rates of the box (context for the roofline)
    res["probes"] = {
        "gather_1KiB_GBs": F.ftlm_peak_probe(F.PEAK_GATHER, 2 << 30, 1024) / 1e9,
        "stream_copy_GBs": F.ftlm_peak_probe(F.PEAK_STREAM, 2 << 30) / 1e9,
        "ffma32_Tflops": 2 * F.ftlm_peak_probe(F.PEAK_FFMA32) / 1e12,
        "dfma64_Tflops": 2 * F.ftlm_peak_probe(F.PEAK_DFMA64) / 1e12,
        "lop3_Tops": F.ftlm_peak_probe(F.PEAK_LOP3) / 1e12,
    }
    return res


def _flip_count(labels, bonds):
    """Admissible s=1/2 ladder flips summed over representatives (antiparallel bonds)."""
    lab = labels.astype(np.uint64)
    total = 0
    for i, j in bonds:
        total += int(np.count_nonzero(((lab >> np.uint64(i)) ^ (lab >> np.uint64(j))) & np.uint64(1)))
    return total


def _kernel_sha():
    import hashlib

    h = hashlib.sha256()
    for name in ("hvp.cuh", "hvp_lane.cuh", "ptx.cuh", "contract.cuh"):
        with open(os.path.join(ROOT, "paper_2607_17429_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_record(dtype_name, mode, workload):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source and workload."""
    sha = _kernel_sha()
    path = os.path.join(ROOT, "profiles", "roofline_traffic.md")
    try:
        for ln in open(path):
            p = ln.split()
            if (len(p) >= 6 and p[0] == "hvp_kernel" and p[1] == dtype_name and p[3] == sha and p[4] == mode
                    and p[5] == workload):
                return float(p[2])
    except OSError:
        pass
    return None


def hv_roofline(prof, dtype_name, flips, n_reps, W, B, esize, mode="search",
                workload="icosidodecahedron_s1/2_M0_all10_B8"):
    """Roofline of the dominant kernel (packed H·v), per launch, HBM bound.

    Search path:  flips * (W*B*e + 20)       [every flipped state's segment, its record and bucket]
                + n_reps * (2*W*B*e + 16)    [the representative's own rows in, its outputs out, its record]
    Table path:   flips * (W*B*e + 8)        [segment and 8-byte entry]
                + n_reps * (2*W*B*e + 24)    [own rows, outputs, record and entry offset]
    against the measured STREAM copy bandwidth (MEASURED_PEAKS.json hbm_gbs).  flips per launch is the
    kernel's own device count while profiling (ftlm_profile.hv_flips), else the count from the labels.
    """
    pk, which = peaks()
    if prof["hv_launches"] == 0:
        return None
    if prof.get("hv_flips"):
        flips = prof["hv_flips"] / prof["hv_launches"]
    t = prof["hv_ms"] / prof["hv_launches"] / 1e3
    seg = W * B * esize
    if mode == "table":
        byt = flips * (seg + 8) + n_reps * (2 * seg + 24)
    else:
        byt = flips * (seg + 20) + n_reps * (2 * seg + 16)
    peak = float(pk["hbm_gbs"]) * 1e9
    return {"bound": "hbm", "achieved": byt / t / 1e9, "peak": peak / 1e9, "unit": "GB/s", "frac": byt / t / peak,
            "traffic": _traffic_record(dtype_name, mode, workload), "algorithmic_per_launch": byt,
            "avg_launch_ms": t * 1e3,
            "flip_path": mode,
            "flips_per_launch": flips,
            "peak_source": f"{which} MEASURED_PEAKS.json hbm_gbs" if which == "measured" else "fallback 6.8 TB/s",
            "kernel_sha": _kernel_sha()}


def _oracle_worker(args):
    """One process of the CPU baseline: label-keyed oracle rows for random representatives (spawned)."""
    seed, budget_s, name, two_s, B = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    from oracle import native
    from oracle.basis import hv_rows_by_label
    from oracle.group import Group
    from workloads import cluster, label_keyed_values

    c = cluster(name)
    N, d = c.n_sites, two_s + 1
    og = Group(c.gens, c.bonds)
    inv = og.element(c.gens[2])
    ir = [i for i, r in enumerate(og.irreps) if r.dim == 5 and r.chars[inv] > 0][0]  # H_g
    rng = np.random.default_rng(seed)
    rows = reps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        batch = []
        while len(batch) < 8:  # uniform over the M = 0 product states (rejection on the digit sum)
            dig = rng.integers(0, d, N)
            if int(dig.sum()) * 2 != N * two_s:
                continue
            lab = int(sum(int(v) * d ** k for k, v in enumerate(dig)))
            batch.append(native.min_rep(N, d, og.perms, lab)[0])
        out = hv_rows_by_label(og, ir, c.bonds, 1.0, two_s, batch,
                               lambda lab, n: label_keyed_values([lab], n, B, 1)[0])
        rows += sum(0 if y is None else y.shape[0] for y in out)
        reps += len(batch)
    return rows, reps, time.perf_counter() - t0


def cpu_baseline(budget_s=10.0, name=None, two_s=None, B=None):
    """The oracle's H·v (FP64, label-keyed rows of the H_g block at M = 0) on every host core, bounded sample;
    the benchmark workload by default."""
    import multiprocessing as mp

    name = name or CLUSTER
    two_s = two_s or TWO_S
    B = B or R
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(1000 + i, budget_s, name, two_s, B) for i in range(cores)])
    wall = time.perf_counter() - t0
    rows = sum(r[0] for r in res)
    reps = sum(r[1] for r in res)
    busy = max(r[2] for r in res)
    return {"value": rows * B / busy / 1e9, "unit": "Gstates/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} random representatives of the H_g block (d=5) of the {name} s={two_s}/2 M=0 sector, "
                      f"B={B} right-hand sides, FP64 label-keyed oracle rows (Eqs. 15-16), {cores} spawned "
                      f"processes x {busy:.1f} s (wall {wall:.1f} s including start-up)"}


def hv_once(flips="search"):
    """The profiling case: one packed H·v over all 10 blocks (FP32, B = 8) and one on the H_g block alone;
    with flips="table" the sector's entry table is built first (one build-mode launch) and both H·v read it."""
    import torch

    from paper_2607_17429_gb300 import build as pb

    pb.build()
    from paper_2607_17429_gb300 import ftlm as F
    from workloads import cluster

    torch.cuda.set_device(0)
    c = cluster(CLUSTER)
    g = F.ftlm_group_init(c.gens, c.bonds)
    sec = F.ftlm_build_sector(g, TWO_S, TWO_M)
    if flips == "table":
        F.ftlm_sector_build_entries(sec)
    mb = F.ftlm_build_multiblock(sec, list(range(10)))
    rows = F.ftlm_multiblock_packed_rows(mb)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    xp = torch.randn(rows, R, device="cuda", generator=gen)
    yp = torch.empty_like(xp)
    F.ftlm_hv_packed(mb, F.F32, R, xp, yp)
    F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
    del xp, yp
    blk = F.ftlm_multiblock_block(mb, 8)
    dim = F.ftlm_multiblock_info(mb)["dims"][8]
    x = torch.randn(dim, R, device="cuda", generator=gen)
    y = torch.empty_like(x)
    F.ftlm_hv(blk, F.F32, R, x, y)
    F.ftlm_basis_check(blk)
    torch.cuda.synchronize()
    print(json.dumps({"hv_once": "ok", "packed_rows": rows, "hg_dim": dim}))


def hv_once_lane(flips="table", two_M=28):
    """The profiling stand-in for the largest single block: one FP32 B = 1 H·v of the s=3/2 dodecahedron's
    H_g block at M = two_M/2 (M = 14: 6.9e7 rows, vectors of 0.27 GB, twice L2; the M = 0 block's table
    of ~200 GB is too large for a capture), on the entry table (one-thread-per-representative kernel) or
    searching.  Prints the kernel's flip count and the algorithmic bytes of the launch."""
    import torch

    from paper_2607_17429_gb300 import build as pb

    pb.build()
    from paper_2607_17429_gb300 import ftlm as F
    from workloads import cluster

    torch.cuda.set_device(0)
    c = cluster("dodecahedron")
    g = F.ftlm_group_init(c.gens, c.bonds)
    info = F.ftlm_group_info(g)
    _, perms = F.ftlm_group_irrep(g)
    inv = int(np.nonzero((perms == c.gens[2]).all(axis=1))[0][0])
    ir = [i for i, d in enumerate(info["dims"]) if d == 5 and info["chars"][i][inv] > 0][0]
    sec = F.ftlm_build_sector(g, 3, two_M)
    n_ent = F.ftlm_sector_build_entries(sec) if flips == "table" else None
    mb = F.ftlm_build_multiblock(sec, [ir])
    rows = F.ftlm_multiblock_packed_rows(mb)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    xp = torch.randn(rows, 1, device="cuda", generator=gen)
    yp = torch.empty_like(xp)
    F.ftlm_profile_reset()
    F.ftlm_profile_enable(True)
    F.ftlm_hv_packed(mb, F.F32, 1, xp, yp)
    torch.cuda.synchronize()
    F.ftlm_profile_enable(False)
    prof = F.ftlm_profile_get()
    F.ftlm_basis_check(F.ftlm_multiblock_block(mb, 0))
    n_reps = F.ftlm_sector_info(sec)["n_reps"]
    fl = prof["hv_flips"] / max(1, prof["hv_launches"])
    seg = 5 * 1 * 4
    alg = fl * (seg + 8) + n_reps * (2 * seg + 24) if flips == "table" else fl * (seg + 20) + n_reps * (2 * seg + 16)
    print(json.dumps({"hv_once": "ok", "two_M": two_M, "flip_path": flips, "n_reps": n_reps, "packed_rows": rows,
                      "entries": n_ent, "flips_per_launch": fl, "algorithmic_per_launch": alg,
                      "hv_ms": prof["hv_ms"]}))


def config5(args):
    """Largest single block: s=3/2 dodecahedron (N=20, I_h), M=0, H_g (3 624 380 734 states, Table 2),
    R=1 Gaussian (seed 4), 60 Lanczos steps, FP32 vectors with FP64 alpha/beta, against an FP64 GPU run."""
    import torch

    from paper_2607_17429_gb300 import build as pb

    pb.build()
    from paper_2607_17429_gb300 import ftlm as F
    from workloads import cluster

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    c = cluster("dodecahedron")
    g = F.ftlm_group_init(c.gens, c.bonds)
    info = F.ftlm_group_info(g)
    _, perms = F.ftlm_group_irrep(g)
    inv = int(np.nonzero((perms == c.gens[2]).all(axis=1))[0][0])
    ir = [i for i, d in enumerate(info["dims"]) if d == 5 and info["chars"][i][inv] > 0][0]
    out = {"metric": METRIC.replace("10 irrep blocks x 8 chains", "1 block x 1 chain"), "unit": "Gstates/s",
           "config": {"workload": "dodecahedron s=3/2 M=0 H_g (D=3624380734), R=1 Gaussian (seed 4), 60 Lanczos "
                      "steps", "cluster": "dodecahedron", "two_s": 3, "two_M": 0, "irrep": "H_g"}}
    t0 = time.perf_counter()
    sec = F.ftlm_build_sector(g, 3, 0, stream)
    blk = F.ftlm_build_block(sec, ir, stream)
    torch.cuda.synchronize()
    out["build_s"] = time.perf_counter() - t0
    dim = F.ftlm_basis_info(blk)["dim"]
    out["dim"] = dim
    out["n_reps"] = F.ftlm_sector_info(sec)["n_reps"]
    # FP32 run on the entry table when it fits beside the three vectors (else the search path);
    # the FP64 run (three 29 GB vectors) always searches
    flips32 = "search"
    if args.flips == "table":
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out["entries"] = F.ftlm_sector_build_entries(sec, stream)
            out["entries_build_s"] = time.perf_counter() - t0
            flips32 = "table"
        except F.FtlmError as e:
            out["entries"] = f"not built: {e}"
    out["config"]["flips_f32"] = FLIP_PATHS[flips32]
    out["config"]["flips_f64"] = FLIP_PATHS["search"]
    res = {}
    for name, dt in (("f32", F.F32), ("f64", F.F64)):
        if dt == F.F64 and flips32 == "table":
            F.ftlm_sector_free_entries(sec)
        F.ftlm_profile_reset()
        F.ftlm_profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        try:
            a, b, st = F.ftlm_lanczos(blk, dt, 1, N_STEPS, 4, 8, F.GAUSS, stream)
        except F.FtlmError as e:  # no room for the vectors beside the table: search path
            if not (dt == F.F32 and flips32 == "table" and e.status == F.ENOMEM):
                raise
            F.ftlm_sector_free_entries(sec)
            flips32 = "search"
            out["config"]["flips_f32"] = FLIP_PATHS[flips32] + f" (the table left no room: {e})"
            torch.cuda.synchronize()
            e0.record(stream)
            a, b, st = F.ftlm_lanczos(blk, dt, 1, N_STEPS, 4, 8, F.GAUSS, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        F.ftlm_profile_enable(False)
        prof = F.ftlm_profile_get()
        ms = e0.elapsed_time(e1)
        th = F.ftlm_thermo([dict(two_M=0, d_gamma=5, dim=dim, alpha=a, beta=b, steps=st)], T_GRID, 1.0, stream)
        res[name] = {"ms": ms, "steps": int(st[0]), "prof": prof, "thermo": th,
                     "hv_ms_per_launch": prof["hv_ms"] / max(1, prof["hv_launches"])}
    f32, f64 = res["f32"], res["f64"]
    # the FTLM step of the FP32 run includes its entry-table build
    t_f32 = f32["ms"] / 1e3 + (out.get("entries_build_s", 0.0) if flips32 == "table" else 0.0)
    out["value"] = dim * f32["steps"] / t_f32 / 1e9
    out["ms_lanczos_f32"] = f32["ms"]
    out["ms_lanczos_f64"] = f64["ms"]
    out["hv_ms_per_launch_f32"] = f32["hv_ms_per_launch"]
    out["hv_ms_per_launch_f64"] = f64["hv_ms_per_launch"]
    wl5 = "dodecahedron_s3/2_M0_Hg_B1"
    out["roofline"] = hv_roofline(f32["prof"], "f32", 0, out["n_reps"], 5, 1, 4, flips32, wl5)
    out["roofline_f64_search"] = hv_roofline(f64["prof"], "f64", 0, out["n_reps"], 5, 1, 8, "search", wl5)
    if not args.no_cpu_baseline:  # the oracle on the host cores: sampled rows of the same block, B = 1
        out["cpu_baseline"] = cpu_baseline(budget_s=10.0, name="dodecahedron", two_s=3, B=1)
    sel = T_GRID >= 0.05
    a32, a64 = f32["thermo"], f64["thermo"]
    out["E0_f32"], out["E0_f64"] = a32[4], a64[4]
    out["mixed_vs_fp64"] = {"dE0_rel": abs(a32[4] - a64[4]) / abs(a64[4]),
                            "max_dC_over_Cmax": float(np.abs(a32[2] - a64[2])[sel].max() / a64[2].max()),
                            "max_dlnZ_rel": float(np.abs((a32[0] - a64[0]) / a64[0]).max()),
                            "note": "one M = 0 block: C(T) of that block alone; chi is identically 0"}
    print(json.dumps(out))


def e0_dodecahedron(args):
    """Cross-check against the paper's ground-state energy of the s=3/2 dodecahedron (Section 4.3:
    E0 = -62.4388 from the M = 0 sector, FP32, 60 steps): every Gamma+- block of the spin-flip
    M = 0 sector (G x Z_2), one FP32 Lanczos chain of `--e0-steps` steps each, on the sector's entry
    table; E0 is the lowest Ritz value over the blocks."""
    import torch

    from paper_2607_17429_gb300 import build as pb

    pb.build()
    from paper_2607_17429_gb300 import ftlm as F
    from workloads import cluster

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    c = cluster("dodecahedron")
    g = F.ftlm_group_init(c.gens, c.bonds)
    t0 = time.perf_counter()
    sec = F.ftlm_build_sector_flip(g, 3, stream)
    n_ent = F.ftlm_sector_build_entries(sec, stream)
    torch.cuda.synchronize()
    out = {"workload": "dodecahedron s=3/2, M=0, G x Z2 (240 elements), all 20 irrep blocks, R=1 Gaussian "
                       f"(seed 4), {args.e0_steps} FP32 Lanczos steps per block, entry table",
           "n_reps": F.ftlm_sector_info(sec)["n_reps"], "entries": n_ent, "prep_s": time.perf_counter() - t0,
           "paper_E0": -62.4388, "blocks": []}
    n_ir = F.ftlm_sector_symmetry(sec)["n_irreps"]
    e0 = None
    for k in range(n_ir):
        blk = F.ftlm_build_block(sec, k, stream)
        dim = F.ftlm_basis_info(blk)["dim"]
        if dim == 0:
            continue
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        a, b, st = F.ftlm_lanczos(blk, F.F32, 1, args.e0_steps, 4, 64 * 0 + k, F.GAUSS, stream)
        th, w = F.ftlm_ritz(a, b, st)
        ek = float(th[0, :st[0]].min())
        out["blocks"].append({"irrep": k, "dim": dim, "E0": ek, "steps": int(st[0]),
                              "s": time.perf_counter() - t1})
        e0 = ek if e0 is None else min(e0, ek)
        del blk
    out["E0"] = e0
    out["dE0_vs_paper"] = e0 - out["paper_E0"]
    out["total_s"] = time.perf_counter() - t0
    print(json.dumps(out))


CONFIG3 = [("cuboctahedron", 1), ("cuboctahedron", 2), ("icosahedron", 3)]


def config3(args):
    """Batched SpMM across uneven blocks: s=1/2 and s=1 cuboctahedron (O_h), s=3/2 icosahedron (I_h); every
    M >= 0 sector x every irrep; R = 24 Rademacher vectors (seed 2), 60 steps, FP32 vectors with FP64
    reductions.  Batched form: per cluster, all sectors as the parts of one launch per kernel, the step loop
    in one CUDA graph, geometry from the autotuner.  Plain form: FP64, one block at a time."""
    import torch

    from paper_2607_17429_gb300 import build as pb

    pb.build()
    from paper_2607_17429_gb300 import ftlm as F
    from workloads import cluster

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    R3, NL3, SEED3 = 24, 60, 2
    F.ftlm_set_autotune(1)
    out = {"metric": "FTLM blocks/h and Gstates/s, batched mixed vs plain FP64 (config 3)", "unit": "blocks/h",
           "config": {"workload": "s=1/2 and s=1 cuboctahedron (O_h), s=3/2 icosahedron (I_h), all M>=0 x all "
                      "irreps, R=24 Rademacher (seed 2), 60 Lanczos steps"}, "clusters": {}}
    tot = {"blocks": 0, "states": 0, "ms_batched": 0.0, "ms_plain64": 0.0}
    for name, two_s in CONFIG3:
        c = cluster(name)
        g = F.ftlm_group_init(c.gens, c.bonds)
        info = F.ftlm_group_info(g)
        n_ir = len(info["dims"])
        N = c.n_sites
        sets, ids, Ms = [], [], []
        for two_M in range(N * two_s % 2, N * two_s + 1, 2):
            sec = F.ftlm_build_sector(g, two_s, two_M, stream)
            sets.append(F.ftlm_build_multiblock(sec, list(range(n_ir)), stream))
            ids.append([64 * two_M + k for k in range(n_ir)])
            Ms.append(two_M)
        dims = [F.ftlm_multiblock_info(m)["dims"] for m in sets]
        n_blocks = sum(1 for dd in dims for d in dd if d > 0)

        def blocks_of(a, b, st):
            return [dict(two_M=Ms[i], d_gamma=int(info["dims"][k]), dim=dims[i][k], alpha=a[i][k], beta=b[i][k],
                         steps=st[i][k]) for i in range(len(sets)) for k in range(n_ir) if dims[i][k] > 0]

        F.ftlm_lanczos_sets(sets, F.F32, R3, NL3, SEED3, ids, F.RADEMACHER, stream)  # warm-up (tuning)
        torch.cuda.synchronize()
        F.ftlm_profile_reset()
        F.ftlm_profile_enable(True)
        t0 = time.perf_counter()
        a, b, st = F.ftlm_lanczos_sets(sets, F.F32, R3, NL3, SEED3, ids, F.RADEMACHER, stream)
        torch.cuda.synchronize()
        ms_b = (time.perf_counter() - t0) * 1e3
        F.ftlm_profile_enable(False)
        prof = F.ftlm_profile_get()
        mixed = F.ftlm_thermo(blocks_of(a, b, st), T_GRID, 1.0, stream)
        states = sum(dims[i][k] * int(st[i][k].sum()) for i in range(len(sets)) for k in range(n_ir))
        # plain form: FP64, one block at a time
        a64 = np.zeros_like(a)
        b64 = np.zeros_like(b)
        s64 = np.zeros_like(st)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, mb in enumerate(sets):
            for k in range(n_ir):
                if dims[i][k] == 0:
                    continue
                blk = F.ftlm_multiblock_block(mb, k)
                a64[i][k], b64[i][k], s64[i][k] = F.ftlm_lanczos(blk, F.F64, R3, NL3, SEED3, ids[i][k], F.RADEMACHER,
                                                                 stream)
        torch.cuda.synchronize()
        ms_p = (time.perf_counter() - t0) * 1e3
        ref = F.ftlm_thermo(blocks_of(a64, b64, s64), T_GRID, 1.0, stream)
        sel = T_GRID >= 0.05
        out["clusters"][f"{name} 2s={two_s}"] = {
            "sectors": len(sets), "blocks": n_blocks, "states_applied": states, "ms_batched_mixed": ms_b,
            "ms_plain_fp64": ms_p, "hv_launches": prof["hv_launches"],
            "hv_ms_per_launch": prof["hv_ms"] / max(1, prof["hv_launches"]),
            "blocks_per_hour_batched": n_blocks / (ms_b / 1e3) * 3600, "blocks_per_hour_plain_fp64":
            n_blocks / (ms_p / 1e3) * 3600,
            "mixed_vs_fp64": {"dE0_rel": abs(mixed[4] - ref[4]) / abs(ref[4]),
                              "max_dC_over_Cmax": float(np.abs(mixed[2] - ref[2])[sel].max() / ref[2].max()),
                              "max_dchi_over_chimax": float(np.abs(mixed[3] - ref[3])[sel].max() / ref[3].max())}}
        tot["blocks"] += n_blocks
        tot["states"] += states
        tot["ms_batched"] += ms_b
        tot["ms_plain64"] += ms_p
    out["value"] = tot["blocks"] / (tot["ms_batched"] / 1e3) * 3600
    out["blocks_per_hour_plain_fp64"] = tot["blocks"] / (tot["ms_plain64"] / 1e3) * 3600
    out["batched_mixed_over_plain_fp64"] = out["value"] / out["blocks_per_hour_plain_fp64"]
    out["gstates_per_s_batched"] = tot["states"] / (tot["ms_batched"] / 1e3) / 1e9
    out["autotune"] = F.ftlm_autotune_report()
    print(json.dumps(out))


FLIP_PATHS = {"table": "entry table: one search pass per step (timed), then every H·v reads it",
              "search": "representative search and lookup inside every H·v"}

CONFIG4 = [("icosahedron", 1), ("icosahedron", 5), ("square:4x4", 1), ("square:4x6", 1), ("cuboctahedron", 1)]


def config4_jobs(F, groups, n_jobs=2000, rate=50.0, seed=3):
    """The serving workload: Poisson arrivals at `rate` per second, each job uniform over the five systems,
    then uniform over that system's M >= 0 sectors and its admissible irreps (real, d <= 5; one-dimensional
    on the square lattices), R uniform over {1, 4, 24}, N_L uniform over 40..60."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_jobs))
    jobs = []
    for i in range(n_jobs):
        sysi = int(rng.integers(len(CONFIG4)))
        name, two_s = CONFIG4[sysi]
        g, N, irreps = groups[sysi]
        two_M = int(rng.choice(np.arange(N * two_s % 2, N * two_s + 1, 2)))
        ir = int(rng.choice(irreps))
        jobs.append(dict(t=float(t[i]), sys=sysi, name=name, two_s=two_s, two_M=two_M, irrep=ir,
                         R=int(rng.choice([1, 4, 24])), n_steps=int(rng.integers(40, 61)), block_id=i))
    return jobs


def config4(args):
    """Serving loop (config 4): 2000 FTLM jobs with Poisson arrivals at 50/s over five systems, admitted
    under a 150 GB HBM cap with resident tables shared across jobs, FP32 vectors with FP64 reductions.
    Reports p50/p99 latency (submission to completion), blocks/h and the plain-FP64 one-job-at-a-time rate
    on a sample of the same jobs."""
    import torch

    from paper_2607_17429_gb300 import build as pb

    pb.build()
    from paper_2607_17429_gb300 import ftlm as F
    from workloads import cluster

    torch.cuda.set_device(0)
    groups = []
    for name, two_s in CONFIG4:
        c = cluster(name)
        g = F.ftlm_group_init(c.gens, c.bonds)
        info = F.ftlm_group_info(g)
        sq = name.startswith("square")
        irreps = [k for k, (d, fs) in enumerate(zip(info["dims"], info["fs"]))
                  if fs == 1 and d <= 5 and (d == 1 or not sq)]
        groups.append((g, c.n_sites, irreps))
    n_jobs = args.jobs
    jobs = config4_jobs(F, groups, n_jobs=n_jobs)
    cap = 150 << 30
    srv = F.Server(cap_bytes=cap, n_workers=args.workers, max_parts=32)
    ids = [None] * n_jobs

    def submitter():
        t0 = time.perf_counter()
        for i, j in enumerate(jobs):
            dt = j["t"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            g = groups[j["sys"]][0]
            ids[i] = srv.submit(g, j["two_s"], j["two_M"], j["irrep"], j["R"], j["n_steps"], 3, j["block_id"],
                                F.GAUSS, F.F32)

    th = threading.Thread(target=submitter)
    t_start = time.perf_counter()
    th.start()
    lat, dims, states, empty, failed, fails = [], [], 0, 0, 0, {}
    t_first, t_last = None, 0.0
    for i in range(n_jobs):
        while ids[i] is None:
            time.sleep(0.001)
        try:
            info, a, b, st = srv.wait(ids[i])
        except F.FtlmError as e:
            failed += 1
            j = jobs[i]
            key = f"status {e.status}: {str(e).split(': ', 2)[-1][:120]}"
            fails.setdefault(key, []).append(f"{j['name']} 2s={j['two_s']} 2M={j['two_M']} irrep={j['irrep']} "
                                             f"R={j['R']}")
            continue
        lat.append(info["t_done"] - info["t_submit"])
        t_first = info["t_submit"] if t_first is None else min(t_first, info["t_submit"])
        t_last = max(t_last, info["t_done"])
        if info["dim"] == 0:
            empty += 1
        dims.append(info["dim"])
        states += int(info["dim"]) * int(st.sum())
    th.join()
    wall = time.perf_counter() - t_start
    stats = srv.stats()
    srv.close()
    lat = np.array(lat)
    makespan = t_last - t_first
    done = len(lat) - empty
    # plain FP64, one job at a time (tables built outside the timed calls), on a sample of the same jobs
    sample = [j for j in jobs[: args.plain_sample]]
    tables = {}
    t_plain, n_plain = 0.0, 0
    for j in sample:
        key = (j["sys"], j["two_M"], j["irrep"])
        if key not in tables:
            tables[key] = F.ftlm_build_basis(groups[j["sys"]][0], j["two_s"], j["two_M"], j["irrep"])
        blk = tables[key]
        if F.ftlm_basis_info(blk)["dim"] == 0:
            continue
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F.ftlm_lanczos(blk, F.F64, j["R"], j["n_steps"], 3, j["block_id"], F.GAUSS)
        t_plain += time.perf_counter() - t0
        n_plain += 1
    out = {"metric": "FTLM serving: p50/p99 job latency and blocks/h (config 4)", "unit": "blocks/h",
           "config": {"workload": "2000 jobs, Poisson arrivals 50/s (seed 3), uniform over s=1/2 and s=5/2 "
                      "icosahedron, 4x4 and 4x6 square lattices, s=1/2 cuboctahedron; random (M, Gamma), "
                      "R in {1,4,24}, N_L in 40..60; 150 GB admission cap; FP32 vectors, FP64 reductions",
                      "n_jobs": n_jobs, "workers": args.workers},
           "value": done / makespan * 3600 if makespan > 0 else None,
           "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                         "max": float(lat.max()), "mean": float(lat.mean())},
           "jobs_done": int(len(lat)), "jobs_failed": failed,
           "failures": {k: {"count": len(v), "first": v[:3]} for k, v in fails.items()},
           "empty_blocks": empty, "makespan_s": makespan,
           "wall_s": wall, "gstates_per_s": states / makespan / 1e9 if makespan > 0 else None,
           "plain_fp64_one_at_a_time": {"jobs": n_plain, "s": t_plain,
                                        "blocks_per_hour": n_plain / t_plain * 3600 if t_plain > 0 else None},
           "server": {k: stats[k] for k in ("waves", "parts", "sectors_built", "sector_hits", "blocks_built",
                                             "block_hits", "evictions", "peak_charged", "resident_table_bytes")}}
    if t_plain > 0 and out["value"]:
        out["served_mixed_over_plain_fp64"] = out["value"] / out["plain_fp64_one_at_a_time"]["blocks_per_hour"]
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flips", default="table", choices=["table", "search"],
                    help="entry table built once per step (the paper's two-phase design) or search in every H·v")
    ap.add_argument("--hv-once", action="store_true",
                    help="one packed 10-block H·v and one H_g-block H·v of the workload, then exit (profiling case)")
    ap.add_argument("--config5", action="store_true",
                    help="the largest single block instead: s=3/2 dodecahedron, M=0, H_g (3.6e9 states), R=1")
    ap.add_argument("--two-M", type=int, default=28,
                    help="with --hv-once --config5: the M sector (2M) of the scaled-down profiling case")
    ap.add_argument("--e0-check", action="store_true",
                    help="cross-check E0 of the s=3/2 dodecahedron against the paper (all M=0 Gamma+- blocks)")
    ap.add_argument("--e0-steps", type=int, default=60)
    ap.add_argument("--config4", action="store_true",
                    help="serving loop: 2000 Poisson-arrival jobs over five systems under a 150 GB cap")
    ap.add_argument("--jobs", type=int, default=2000)
    ap.add_argument("--workers", type=int, default=3)
    ap.add_argument("--plain-sample", type=int, default=200)
    ap.add_argument("--config3", action="store_true",
                    help="batched small blocks instead: every M>=0 sector x irrep of three clusters, R=24 Rademacher")
    args = ap.parse_args()
    if args.hv_once:
        if args.config5:
            hv_once_lane(args.flips, args.two_M)
        else:
            hv_once(args.flips)
        return
    if args.config5:
        config5(args)
        return
    if args.config4:
        config4(args)
        return
    if args.e0_check:
        e0_dodecahedron(args)
        return
    if args.config3:
        config3(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        K = max(1, args.steps)
        for _ in range(max(0, args.warmup)):
            cpu_baseline(budget_s=2.0)
        t0 = time.perf_counter()
        vals = [cpu_baseline(budget_s=10.0) for _ in range(K)]
        ms_step = (time.perf_counter() - t0) * 1e3 / K
        v = float(np.mean([b["value"] for b in vals]))
        cb = dict(vals[-1])
        cb["value"] = v
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "Gstates/s", "n_gpus": args.gpus,
                          "steps": K, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": WORKLOAD, "sample": "bounded oracle sample per step"},
                          "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": "Gstates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank != 0:
        return
    prof = res["prof"]
    esize = 4 if args.dtype == "f32" else 8
    rl = hv_roofline(prof, args.dtype, res["flips"], res["n_reps"], res["W"], R, esize, args.flips)
    line = {
        "metric": METRIC, "value": res["value"], "unit": "Gstates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_all"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "cluster": CLUSTER, "two_s": TWO_S, "two_M": TWO_M, "R": R,
                   "lanczos_steps": N_STEPS, "blocks": len(res["dims"]), "flips": FLIP_PATHS[args.flips],
                   "precision": "FP32 vectors, FP64 alpha/beta"
                   if args.dtype == "f32" else "FP64", "l2": "inputs larger than L2 (three packed [41.4M][8] "
                   "vectors of 1.3 GB each in FP32)", "parallelism": f"replicas{world}"},
        "blocks_per_hour": len(res["dims"]) * args.steps / (res["ms_all"] / 1e3) * 3600.0 * world,
        "gpu_launches": int(prof["kernel_launches"]),
        "hv_launches": int(prof["hv_launches"]),
        "hv_ms_per_launch": prof["hv_ms"] / max(1, prof["hv_launches"]),
        "roofline": rl,
        "E0": res["out"][4],
        "e2e": res["e2e"],
        "clocks": res["clocks"],
        "fp64": res["fp64"],
        "fp16_storage": res.get("fp16_storage"),
        "other_flip_path": res.get("other_flip_path"),
        "probes": res["probes"],
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
