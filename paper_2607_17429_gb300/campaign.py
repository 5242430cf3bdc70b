"""FTLM campaigns over (M, Gamma) blocks with per-block checkpoints.

The natural unit of a campaign is the block (Section 4.3 runs the dodecahedron sector by
sector and irrep by irrep): every finished block writes one small file with its Lanczos
coefficients and the numbers Eqs. 5-7 and 14 need (2M, weight, dimension, R), so the
thermal sums can be recomputed from the files alone, and a rerun of an interrupted
campaign skips the blocks whose files exist and belong to the same campaign.  Files are
written to a temporary name and renamed, so a crash leaves either a complete file or none.

A campaign is described by a JSON file (``CampaignConfig``); ``python -m
paper_2607_17429_gb300.campaign CONFIG.json`` runs or resumes it and prints the thermal
sums as one JSON line.  Every block runs through the library (ftlm_build_sector /
ftlm_build_block / ftlm_lanczos); this module only orders the work, names the files and
checks them.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import sys
import time
import zipfile

import numpy as np

DTYPES = {"f64": 0, "f32": 1, "f16": 2}
RNGS = {"gauss": 0, "rademacher": 1}


def default_temperatures():
    """200 log-spaced temperatures T_i = 0.02 * 5000^(i/199) (J = k_B = 1)."""
    return (0.02 * 5000.0 ** (np.arange(200) / 199.0)).tolist()


@dataclasses.dataclass
class CampaignConfig:
    """One campaign: a cluster (a built-in name, or site-permutation generators and bonds), a spin,
    the M sectors and irreps to run (all M >= 0 and all irreps by default), and the Lanczos setup."""

    out_dir: str
    cluster: str | None = None
    gens: list | None = None
    bonds: list | None = None
    J: float = 1.0
    two_s: int = 1
    two_M: list | None = None
    irreps: list | None = None
    flip: bool = False  # the M = 0 sector under G x Z_2 (Section 2.2), its Gamma+- blocks only
    R: int = 8
    n_steps: int = 60
    seed: int = 0
    dtype: str = "f32"
    rng: str = "gauss"
    T: list | None = None
    g: float = 1.0

    @classmethod
    def from_json(cls, path_or_text: str) -> "CampaignConfig":
        text = path_or_text
        if not path_or_text.lstrip().startswith("{"):
            with open(path_or_text) as f:
                text = f.read()
        d = json.loads(text)
        unknown = set(d) - {f.name for f in dataclasses.fields(cls)}
        if unknown:
            raise ValueError(f"unknown campaign keys: {sorted(unknown)}")
        cfg = cls(**d)
        cfg.validate()
        return cfg

    def to_json(self) -> str:
        return json.dumps(dataclasses.asdict(self), indent=1)

    def validate(self) -> None:
        if (self.cluster is None) == (self.gens is None):
            raise ValueError("give either a built-in cluster name or gens + bonds")
        if self.gens is not None and self.bonds is None:
            raise ValueError("gens need bonds")
        if self.dtype not in DTYPES or self.rng not in RNGS:
            raise ValueError("dtype must be f64, f32 or f16 and rng gauss or rademacher")
        if self.R < 1 or not 1 <= self.n_steps <= 512 or self.two_s < 1:
            raise ValueError("R >= 1, 1 <= n_steps <= 512, two_s >= 1")
        if self.flip and self.two_M not in (None, [0]):
            raise ValueError("the spin-flip campaign is the M = 0 sector only")

    def key(self) -> str:
        """Identity of the campaign's blocks: a file written under another key is recomputed."""
        d = {k: getattr(self, k) for k in ("cluster", "gens", "bonds", "J", "two_s", "flip", "R", "n_steps",
                                            "seed", "dtype", "rng")}
        return hashlib.sha256(json.dumps(d, sort_keys=True).encode()).hexdigest()[:20]


def block_id(two_M: int, irrep: int) -> int:
    """Philox key word 1 of a block's start vectors (the same numbering as the tests)."""
    return 64 * two_M + irrep


def block_path(out_dir: str, two_M: int, irrep: int) -> str:
    return os.path.join(out_dir, f"block_M{two_M:03d}_G{irrep:03d}.npz")


def save_block(path: str, rec: dict) -> None:
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        np.savez(f, **{k: np.asarray(v) for k, v in rec.items()})
    os.replace(tmp, path)


def load_block(path: str, key: str) -> dict | None:
    """The block's record, or None when the file is missing, unreadable or from another campaign."""
    try:
        with np.load(path, allow_pickle=False) as z:
            rec = {k: z[k] for k in z.files}
    except (OSError, ValueError, EOFError, KeyError, zipfile.BadZipFile):
        return None
    try:
        if str(rec["key"]) != key:
            return None
        R = int(rec["R"])
        a, b, st = rec["alpha"], rec["beta"], rec["steps"]
        if a.shape[0] != R or b.shape != a.shape or st.shape != (R,) or int(st.max(initial=0)) > a.shape[1]:
            return None
    except KeyError:
        return None
    return rec


class LibraryRunner:
    """Runs one block through the library: sectors are built once per M and reused across irreps."""

    def __init__(self, cfg: CampaignConfig):
        from . import build

        build.build()
        from . import ftlm as F

        self.F = F
        self.cfg = cfg
        if cfg.cluster is not None:
            self.group = F.ftlm_group_builtin(cfg.cluster)
        else:
            self.group = F.ftlm_group_init(np.asarray(cfg.gens, dtype=np.int32), np.asarray(cfg.bonds, dtype=np.int32),
                                           J=cfg.J)
        info = F.ftlm_group_info(self.group)
        self.n_sites = info["n_sites"]
        self.weights = info["weights"]
        self._sector = (None, None)

    def blocks(self) -> list:
        """(2M, irrep) of every block the campaign covers, in run order."""
        cfg = self.cfg
        if cfg.flip:
            n_ir = 2 * len(self.weights)
            return [(0, k) for k in (cfg.irreps if cfg.irreps is not None else range(n_ir))]
        Ms = cfg.two_M
        if Ms is None:
            N = self.n_sites
            Ms = list(range(N * cfg.two_s % 2, N * cfg.two_s + 1, 2))
        irs = cfg.irreps if cfg.irreps is not None else range(len(self.weights))
        return [(m, k) for m in Ms for k in irs]

    def sector(self, two_M: int):
        if self._sector[0] != two_M:
            self._sector = (None, None)
            F = self.F
            sec = F.ftlm_build_sector_flip(self.group, self.cfg.two_s) if self.cfg.flip else \
                F.ftlm_build_sector(self.group, self.cfg.two_s, two_M)
            self._sector = (two_M, sec)
        return self._sector[1]

    def weight(self, irrep: int) -> int:
        return int(self.weights[irrep // 2 if self.cfg.flip else irrep])

    def __call__(self, two_M: int, irrep: int) -> dict:
        cfg, F = self.cfg, self.F
        blk = F.ftlm_build_block(self.sector(two_M), irrep)
        dim = int(F.ftlm_basis_info(blk)["dim"])
        if dim == 0:
            a = np.zeros((cfg.R, cfg.n_steps))
            return dict(alpha=a, beta=a.copy(), steps=np.zeros(cfg.R, dtype=np.int32), dim=0)
        a, b, st = F.ftlm_lanczos(blk, DTYPES[cfg.dtype], cfg.R, cfg.n_steps, cfg.seed, block_id(two_M, irrep),
                                  RNGS[cfg.rng])
        return dict(alpha=a, beta=b, steps=st, dim=dim)


def run(cfg: CampaignConfig, runner=None, log=None) -> list:
    """Run or resume the campaign; returns the records of every block in run order.

    runner(two_M, irrep) -> {alpha, beta, steps, dim} and runner.blocks(), runner.weight(irrep) default to
    the library.  An exception from the runner propagates after the finished blocks are on disk."""
    cfg.validate()
    runner = runner if runner is not None else LibraryRunner(cfg)
    os.makedirs(cfg.out_dir, exist_ok=True)
    key = cfg.key()
    with open(os.path.join(cfg.out_dir, "campaign.json"), "w") as f:
        f.write(cfg.to_json())
    out = []
    for two_M, irrep in runner.blocks():
        path = block_path(cfg.out_dir, two_M, irrep)
        rec = load_block(path, key)
        if rec is None:
            t0 = time.perf_counter()
            res = runner(two_M, irrep)
            rec = dict(key=key, two_M=two_M, irrep=irrep, weight=runner.weight(irrep), R=cfg.R,
                       dim=int(res["dim"]), alpha=np.asarray(res["alpha"], dtype=np.float64),
                       beta=np.asarray(res["beta"], dtype=np.float64), steps=np.asarray(res["steps"], dtype=np.int32),
                       seconds=time.perf_counter() - t0)
            save_block(path, rec)
            rec = load_block(path, key)
            if log:
                log(f"block 2M={two_M} irrep={irrep} dim={int(rec['dim'])} {float(rec['seconds']):.3f} s")
        elif log:
            log(f"block 2M={two_M} irrep={irrep} from its checkpoint")
        out.append(rec)
    return out


def thermo(cfg: CampaignConfig, records: list) -> dict:
    """Eqs. 5-7 and 14 over the records (blocks of dimension 0 contribute nothing), on the GPU."""
    from . import build

    build.build()
    from . import ftlm as F

    blocks = [dict(two_M=int(r["two_M"]), d_gamma=int(r["weight"]), dim=int(r["dim"]), alpha=r["alpha"],
                   beta=r["beta"], steps=r["steps"]) for r in records if int(r["dim"]) > 0]
    T = np.asarray(cfg.T if cfg.T is not None else default_temperatures(), dtype=np.float64)
    lnZ, E, C, chi, E0 = F.ftlm_thermo(blocks, T, cfg.g)
    return dict(T=T.tolist(), lnZ=lnZ.tolist(), E=E.tolist(), C=C.tolist(), chi=chi.tolist(), E0=E0)


def baseline_configs(out_root: str) -> dict:
    """Campaign descriptions of the five benchmark workloads (cluster, s, sectors, R, seed, steps, precision)."""
    return {
        "config1_icosahedron_s1/2": CampaignConfig(out_dir=os.path.join(out_root, "config1"), cluster="icosahedron",
                                                   two_s=1, R=4, n_steps=30, seed=0, dtype="f64"),
        "config2_icosidodecahedron_s1/2_M0": CampaignConfig(out_dir=os.path.join(out_root, "config2"),
                                                            cluster="icosidodecahedron", two_s=1, two_M=[0], R=8,
                                                            n_steps=60, seed=1, dtype="f32"),
        "config3_cuboctahedron_s1/2": CampaignConfig(out_dir=os.path.join(out_root, "config3a"),
                                                     cluster="cuboctahedron", two_s=1, R=24, n_steps=60, seed=2,
                                                     dtype="f32", rng="rademacher"),
        "config3_cuboctahedron_s1": CampaignConfig(out_dir=os.path.join(out_root, "config3b"),
                                                   cluster="cuboctahedron", two_s=2, R=24, n_steps=60, seed=2,
                                                   dtype="f32", rng="rademacher"),
        "config3_icosahedron_s3/2": CampaignConfig(out_dir=os.path.join(out_root, "config3c"), cluster="icosahedron",
                                                   two_s=3, R=24, n_steps=60, seed=2, dtype="f32",
                                                   rng="rademacher"),
        "config5_dodecahedron_s3/2_M0_Hg": CampaignConfig(out_dir=os.path.join(out_root, "config5"),
                                                          cluster="dodecahedron", two_s=3, two_M=[0], irreps=[8],
                                                          R=1, n_steps=60, seed=4, dtype="f32"),
    }


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description="Run or resume an FTLM campaign described by a JSON file.")
    ap.add_argument("config", nargs="?", help="campaign JSON (see CampaignConfig)")
    ap.add_argument("--thermo-only", action="store_true", help="thermal sums from the checkpoints, no new blocks")
    ap.add_argument("--write-baseline-configs", metavar="DIR",
                    help="write the benchmark workloads' campaign JSON files into DIR and exit")
    args = ap.parse_args(argv)
    if args.write_baseline_configs:
        os.makedirs(args.write_baseline_configs, exist_ok=True)
        for name, cfg in baseline_configs(os.path.join(args.write_baseline_configs, "runs")).items():
            with open(os.path.join(args.write_baseline_configs, name.replace("/", "_") + ".json"), "w") as f:
                f.write(cfg.to_json())
        return 0
    if not args.config:
        ap.error("a campaign JSON is required")
    cfg = CampaignConfig.from_json(args.config)
    if args.thermo_only:
        key = cfg.key()
        names = sorted(p for p in os.listdir(cfg.out_dir) if p.startswith("block_") and p.endswith(".npz"))
        records = [r for r in (load_block(os.path.join(cfg.out_dir, p), key) for p in names) if r is not None]
    else:
        records = run(cfg, log=lambda s: print(s, file=sys.stderr))
    res = thermo(cfg, records)
    res["blocks"] = len(records)
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
