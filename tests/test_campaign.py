"""Campaign driver: per-block checkpoints, resume after a failure, JSON configs.

Host-side fault injection (no GPU fault is ever provoked): a fake block runner raises on a
chosen block, as a failing allocation or a killed job would; the finished blocks are on disk,
the rerun computes only the missing ones, and its records equal an uninterrupted run's.
Corrupt or foreign checkpoint files are recomputed, never trusted.  The GPU test runs a real
campaign through the library, interrupts it, resumes it and compares the thermal sums.
"""
import json
import os

import numpy as np
import pytest

from paper_2607_17429_gb300 import campaign as C


class FakeRunner:
    """Deterministic stand-in for the library: coefficients drawn from the block id."""

    def __init__(self, cfg, fail_at=None, exc=RuntimeError):
        self.cfg, self.fail_at, self.exc = cfg, fail_at, exc
        self.calls = []

    def blocks(self):
        return [(m, k) for m in (0, 2, 4) for k in range(4)]

    def weight(self, irrep):
        return [1, 1, 2, 3][irrep]

    def __call__(self, two_M, irrep):
        if self.fail_at is not None and len(self.calls) == self.fail_at:
            raise self.exc("injected failure")
        self.calls.append((two_M, irrep))
        rng = np.random.default_rng(C.block_id(two_M, irrep))
        R, n = self.cfg.R, self.cfg.n_steps
        st = rng.integers(1, n + 1, R).astype(np.int32)
        return dict(alpha=rng.standard_normal((R, n)), beta=np.abs(rng.standard_normal((R, n))), steps=st,
                    dim=int(rng.integers(1, 1000)))


def _cfg(tmp_path, **kw):
    d = dict(out_dir=str(tmp_path / "run"), cluster="icosahedron", two_s=1, R=3, n_steps=7, seed=5, dtype="f64")
    d.update(kw)
    return C.CampaignConfig(**d)


def _same(ra, rb):
    assert len(ra) == len(rb)
    for a, b in zip(ra, rb):
        for k in ("two_M", "irrep", "weight", "R", "dim"):
            assert int(a[k]) == int(b[k])
        for k in ("alpha", "beta", "steps"):
            assert np.array_equal(a[k], b[k])


def test_resume_after_injected_failure(tmp_path):
    clean = C.run(_cfg(tmp_path, out_dir=str(tmp_path / "clean")), FakeRunner(_cfg(tmp_path)))
    cfg = _cfg(tmp_path)
    r1 = FakeRunner(cfg, fail_at=5, exc=MemoryError)
    with pytest.raises(MemoryError):
        C.run(cfg, r1)
    done = sorted(p for p in os.listdir(cfg.out_dir) if p.endswith(".npz"))
    assert len(done) == 5 and not [p for p in os.listdir(cfg.out_dir) if ".tmp" in p]
    r2 = FakeRunner(cfg)
    resumed = C.run(cfg, r2)
    assert r2.calls == r1.blocks()[5:]  # only the missing blocks run
    _same(resumed, clean)
    r3 = FakeRunner(cfg)
    _same(C.run(cfg, r3), clean)  # everything from checkpoints
    assert r3.calls == []


def test_corrupt_and_foreign_checkpoints_are_recomputed(tmp_path):
    cfg = _cfg(tmp_path)
    ref = C.run(cfg, FakeRunner(cfg))
    p0 = C.block_path(cfg.out_dir, 0, 1)
    with open(p0, "r+b") as f:  # truncated file
        f.truncate(40)
    other = _cfg(tmp_path, seed=6)  # a file of another campaign in the same directory
    rec = C.load_block(C.block_path(cfg.out_dir, 2, 3), cfg.key())
    rec["key"] = np.asarray(other.key())
    C.save_block(C.block_path(cfg.out_dir, 2, 3), rec)
    r = FakeRunner(cfg)
    _same(C.run(cfg, r), ref)
    assert r.calls == [(0, 1), (2, 3)]


def test_config_json_round_trip_and_validation(tmp_path):
    cfg = _cfg(tmp_path, two_M=[0, 2], irreps=[1, 4], rng="rademacher", dtype="f16")
    back = C.CampaignConfig.from_json(cfg.to_json())
    assert back == cfg and back.key() == cfg.key()
    assert _cfg(tmp_path, seed=9).key() != cfg.key()
    for bad in (dict(cluster=None), dict(dtype="bf16"), dict(n_steps=0), dict(flip=True, two_M=[2])):
        with pytest.raises(ValueError):
            C.CampaignConfig(**{**dataclass_dict(_cfg(tmp_path)), **bad}).validate()
    with pytest.raises(ValueError):
        C.CampaignConfig.from_json(json.dumps({"out_dir": "x", "cluster": "icosahedron", "bogus": 1}))


def dataclass_dict(cfg):
    import dataclasses

    return dataclasses.asdict(cfg)


def test_baseline_config_files(tmp_path):
    assert C.main(["--write-baseline-configs", str(tmp_path)]) == 0
    files = sorted(os.listdir(tmp_path))
    assert len([f for f in files if f.endswith(".json")]) == 6
    for f in files:
        if f.endswith(".json"):
            cfg = C.CampaignConfig.from_json(str(tmp_path / f))
            assert cfg.cluster in ("icosahedron", "icosidodecahedron", "cuboctahedron", "dodecahedron")
    c5 = C.CampaignConfig.from_json(str(tmp_path / "config5_dodecahedron_s3_2_M0_Hg.json"))
    assert (c5.two_s, c5.two_M, c5.R, c5.seed, c5.n_steps) == (3, [0], 1, 4, 60)


@pytest.mark.gpu
def test_library_campaign_interrupted_and_resumed(tmp_path):
    """icosahedron s=1/2, every M >= 0 and irrep, R = 2, 20 FP64 steps: a campaign stopped after six
    blocks and resumed gives the same coefficients, bit for bit, and the same thermal sums."""
    cfg = _cfg(tmp_path, R=2, n_steps=20, seed=3, out_dir=str(tmp_path / "a"))
    full = C.run(cfg)
    th_full = C.thermo(cfg, full)

    class Stop(C.LibraryRunner):
        def __call__(self, two_M, irrep):
            if getattr(self, "n", 0) == 6:
                raise KeyboardInterrupt
            self.n = getattr(self, "n", 0) + 1
            return super().__call__(two_M, irrep)

    cfg_b = _cfg(tmp_path, R=2, n_steps=20, seed=3, out_dir=str(tmp_path / "b"))
    with pytest.raises(KeyboardInterrupt):
        C.run(cfg_b, Stop(cfg_b))
    resumed = C.run(cfg_b)
    _same(resumed, full)
    th = C.thermo(cfg_b, resumed)
    assert th["lnZ"] == th_full["lnZ"] and th["C"] == th_full["C"] and th["E0"] == th_full["E0"]
    assert sum(int(r["dim"]) * int(r["weight"]) * (2 if int(r["two_M"]) else 1) for r in full) == 2 ** 12
