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

    def step_multi(grp, dt):
        """Batched form: all 10 irrep blocks through one packed H·v launch per Lanczos step."""
        sec = F.ftlm_build_sector(grp, TWO_S, TWO_M, stream)
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
    ms_all = ms
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_all = float(t.item())
    value = states * world / (ms_all / 1e3) / 1e9  # replicas: every rank runs the same workload
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
    for name in ("hvp.cuh", "ptx.cuh", "contract.cuh"):
        with open(os.path.join(ROOT, "paper_2607_17429_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_record(dtype_name):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    sha = _kernel_sha()
    path = os.path.join(ROOT, "profiles", "roofline_traffic.md")
    try:
        for ln in open(path):
            p = ln.split()
            if len(p) >= 4 and p[0] == "hvp_kernel" and p[1] == dtype_name and p[3] == sha:
                return float(p[2])
    except OSError:
        pass
    return None


def hv_roofline(prof, dtype_name, flips, n_reps, W, B, esize):
    """Roofline of the dominant kernel (packed H·v), per launch, HBM bound.

    Algorithmic bytes = flips * (W*B*e + 20)   [every flipped state's segment, its record and bucket]
                      + n_reps * (2*W*B*e + 16) [the representative's own rows in, its outputs out, its record]
    against the measured STREAM copy bandwidth (MEASURED_PEAKS.json hbm_gbs).
    """
    pk, which = peaks()
    if prof["hv_launches"] == 0:
        return None
    t = prof["hv_ms"] / prof["hv_launches"] / 1e3
    seg = W * B * esize
    byt = flips * (seg + 20) + n_reps * (2 * seg + 16)
    peak = float(pk["hbm_gbs"]) * 1e9
    return {"bound": "hbm", "achieved": byt / t / 1e9, "peak": peak / 1e9, "unit": "GB/s", "frac": byt / t / peak,
            "traffic": _traffic_record(dtype_name), "algorithmic_per_launch": byt, "avg_launch_ms": t * 1e3,
            "peak_source": f"{which} MEASURED_PEAKS.json hbm_gbs" if which == "measured" else "fallback 6.8 TB/s",
            "kernel_sha": _kernel_sha()}


def _oracle_worker(args):
    """One process of the CPU baseline: label-keyed oracle rows for random representatives (spawned)."""
    seed, budget_s = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    from oracle import native
    from oracle.basis import hv_rows_by_label
    from oracle.group import Group
    from workloads import cluster, label_keyed_values

    c = cluster(CLUSTER)
    og = Group(c.gens, c.bonds)
    inv = og.element(c.gens[2])
    ir = [i for i, r in enumerate(og.irreps) if r.dim == 5 and r.chars[inv] > 0][0]  # H_g
    rng = np.random.default_rng(seed)
    rows = reps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        batch = []
        for _ in range(8):
            bits = rng.permutation(np.r_[np.ones(15, dtype=np.int64), np.zeros(15, dtype=np.int64)])
            lab = int(sum(int(v) << k for k, v in enumerate(bits)))
            batch.append(native.min_rep(30, 2, og.perms, lab)[0])
        out = hv_rows_by_label(og, ir, c.bonds, 1.0, TWO_S, batch,
                               lambda lab, n: label_keyed_values([lab], n, R, 1)[0])
        rows += sum(0 if y is None else y.shape[0] for y in out)
        reps += len(batch)
    return rows, reps, time.perf_counter() - t0


def cpu_baseline(budget_s=10.0):
    """The oracle's H·v (FP64, label-keyed rows of the H_g block, B = 8) on every host core, bounded sample."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(1000 + i, budget_s) for i in range(cores)])
    wall = time.perf_counter() - t0
    rows = sum(r[0] for r in res)
    reps = sum(r[1] for r in res)
    busy = max(r[2] for r in res)
    return {"value": rows * R / busy / 1e9, "unit": "Gstates/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} random representatives of the H_g block (d=5) of the icosidodecahedron M=0 sector, "
                      f"B={R} right-hand sides, FP64 label-keyed oracle rows (Eqs. 15-16), {cores} spawned "
                      f"processes x {busy:.1f} s (wall {wall:.1f} s including start-up)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
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
    rl = hv_roofline(prof, args.dtype, res["flips"], res["n_reps"], res["W"], R, esize)
    line = {
        "metric": METRIC, "value": res["value"], "unit": "Gstates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_all"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "cluster": CLUSTER, "two_s": TWO_S, "two_M": TWO_M, "R": R,
                   "lanczos_steps": N_STEPS, "blocks": len(res["dims"]), "precision": "FP32 vectors, FP64 alpha/beta"
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
        "probes": res["probes"],
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
