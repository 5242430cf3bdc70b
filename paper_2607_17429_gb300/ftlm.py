"""Thin ctypes binding of libftlm.so (the C ABI in include/ftlm.h).

Functions keep the C names; this module only marshals arguments (numpy arrays
for host buffers, integer device pointers / torch tensors for device buffers)
and turns a non-zero ftlm_status into ``FtlmError``.  Every step of the
computation runs in the library.  Importing fails loudly when the library has
not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOTGROUP, EBONDS, EIRREP, EUNSUPPORTED, ENOMEM, ECUDA, ETIMEOUT, EINTERNAL = range(10)
F64, F32, F16 = 0, 1, 2
GAUSS, RADEMACHER = 0, 1

LIB_PATH = _build.LIB
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libftlm.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                      f"python -m paper_2607_17429_gb300.build")
_lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I = ctypes.c_int
_U64 = ctypes.c_uint64


class FtlmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ftlm status {status}: {msg}")
        self.status = status


class ftlm_profile(ctypes.Structure):
    _fields_ = [("kernel_launches", _U64), ("hv_launches", _U64), ("hv_ms", ctypes.c_double), ("hv_rows", _U64),
                ("hv_flips", _U64)]


class ftlm_block(ctypes.Structure):
    _fields_ = [("two_M", _I), ("d_gamma", _I), ("dim", _U64), ("R", _I), ("ld", _I),
                ("steps_done", _P), ("alpha", _P), ("beta", _P)]


class ftlm_job(ctypes.Structure):
    _fields_ = [("group", _P), ("two_s", _I), ("two_M", _I), ("irrep", _I), ("R", _I), ("n_steps", _I),
                ("seed", _U64), ("block_id", _U64), ("rng", _I), ("dtype", _I)]


class ftlm_job_info(ctypes.Structure):
    _fields_ = [("status", _I), ("d_gamma", _I), ("dim", _U64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class ftlm_server_stats(ctypes.Structure):
    _fields_ = [(n, _U64) for n in ("submitted", "completed", "failed", "waves", "parts", "sectors_built",
                                    "sector_hits", "blocks_built", "block_hits", "evictions")] + \
               [(n, ctypes.c_size_t) for n in ("cap", "charged", "peak_charged", "resident_table_bytes")] + \
               [(n, _I) for n in ("queued", "ready", "running_waves")]


_SIGS = {
    "ftlm_group_init": [_I, _I, _P, _I, _P, ctypes.c_double, _P],
    "ftlm_group_builtin": [ctypes.c_char_p, _P],
    "ftlm_group_info": [_P, _P, _P, _P, _P, _P, _P],
    "ftlm_group_weights": [_P, _P],
    "ftlm_group_irrep": [_P, _I, _P, _P],
    "ftlm_group_bonds": [_P, _P, _P, _P],
    "ftlm_group_set_irreps": [_P, _I, _P, _P],
    "ftlm_build_sector": [_P, _I, _I, _P, _P],
    "ftlm_sector_info": [_P, _P, _P, _P],
    "ftlm_sector_export": [_P, _P, _P],
    "ftlm_build_block": [_P, _I, _P, _P],
    "ftlm_build_basis": [_P, _I, _I, _I, _P, _P],
    "ftlm_basis_info": [_P, _P, _P, _P],
    "ftlm_basis_export": [_P, _P, _P, _P, _P],
    "ftlm_basis_check": [_P, _P],
    "ftlm_hv": [_P, _I, _I, _P, _P, _P],
    "ftlm_lanczos": [_P, _I, _I, _I, _U64, _U64, _I, _P, _P, _P, _P],
    "ftlm_ritz": [_I, _I, _P, _P, _P, _P, _P, _P],
    "ftlm_thermo": [_I, _P, _I, _P, ctypes.c_double, _P, _P, _P, _P, _P, _P],
    "ftlm_build_multiblock": [_P, _I, _P, _P, _P],
    "ftlm_multiblock_info": [_P, _P, _P, _P],
    "ftlm_multiblock_block": [_P, _I, _P],
    "ftlm_hv_multi": [_P, _I, _I, _P, _P, _P],
    "ftlm_lanczos_multi": [_P, _I, _I, _I, _U64, _P, _I, _P, _P, _P, _P],
    "ftlm_lanczos_sets": [_I, _P, _I, _I, _I, _U64, _P, _I, _P, _P, _P, _P],
    "ftlm_thermo_noalloc": [_I, _I, _P, _P, _P, _P, _P, _I, _P, ctypes.c_double, _P, _P, _P],
    "ftlm_peak_probe": [_I, _U64, _I, _P, _P],
    "ftlm_multiblock_packed_rows": [_P, _P],
    "ftlm_multiblock_pack": [_P, _I, _I, _P, _P, _P],
    "ftlm_multiblock_unpack": [_P, _I, _I, _P, _P, _P],
    "ftlm_hv_packed": [_P, _I, _I, _P, _P, _P],
    "ftlm_set_wait_limit": [_U64],
    "ftlm_set_autotune": [_I],
    "ftlm_autotune_report": [_P, ctypes.c_size_t],
    "ftlm_fill_label_keyed": [_P, _I, _I, _U64, _P, _P],
    "ftlm_basis_rows": [_P, _I, _P, _P, _P, _P],
    "ftlm_build_sector_flip": [_P, _I, _P, _P],
    "ftlm_sector_symmetry": [_P, _P, _P, _P],
    "ftlm_sector_build_entries": [_P, _P, _P],
    "ftlm_sector_free_entries": [_P],
    "ftlm_server_create": [ctypes.c_size_t, _I, _I, _P],
    "ftlm_server_submit": [_P, _P, _P],
    "ftlm_server_wait": [_P, _U64, ctypes.c_double, _P, _P, _P, _P],
    "ftlm_server_stats_get": [_P, _P],
    "ftlm_profile_enable": [_I],
    "ftlm_profile_reset": [],
    "ftlm_profile_get": [_P],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
for _name in ("ftlm_group_free", "ftlm_sector_free", "ftlm_basis_free", "ftlm_multiblock_free", "ftlm_server_free"):
    getattr(_lib, _name).argtypes = [_P]
    getattr(_lib, _name).restype = None
_lib.ftlm_last_error.restype = ctypes.c_char_p
_lib.ftlm_last_error.argtypes = []

EXPORTED = sorted(list(_SIGS) + ["ftlm_group_free", "ftlm_sector_free", "ftlm_basis_free", "ftlm_multiblock_free",
                                  "ftlm_server_free", "ftlm_last_error"])


def _check(st):
    if st != OK:
        raise FtlmError(st, _lib.ftlm_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):  # torch tensor
        return a.data_ptr()
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev(a, dtype=None, numel=None, what="array"):
    """Device address of a caller-owned array: a raw address (int, unchecked) or a CUDA tensor, checked to be
    on a GPU, contiguous, of the element type (a torch dtype name, e.g. "float32") and at least numel long."""
    if a is None or isinstance(a, int):
        return a
    if not hasattr(a, "data_ptr") or not hasattr(a, "is_cuda"):
        raise TypeError(f"{what}: expected a CUDA tensor or a device address (int), got {type(a).__name__}")
    if not a.is_cuda:
        raise ValueError(f"{what}: tensor is on {a.device}, not on a CUDA device")
    if not a.is_contiguous():
        raise ValueError(f"{what}: tensor is not contiguous")
    if dtype is not None and str(a.dtype) != "torch." + dtype:
        raise TypeError(f"{what}: element type {a.dtype}, expected torch.{dtype}")
    if numel is not None and a.numel() < numel:
        raise ValueError(f"{what}: {a.numel()} elements, at least {numel} needed")
    return a.data_ptr()


def _vt(dtype):
    return {F32: "float32", F64: "float64", F16: "float16"}.get(dtype)


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def ftlm_last_error() -> str:
    return _lib.ftlm_last_error().decode()


# ---------------------------------------------------------------- group


class Group:
    """Owning handle of an ftlm_group."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.ftlm_group_free(self._h)
            self._h = None


def ftlm_group_init(gens, bonds, J=1.0) -> Group:
    gens = np.ascontiguousarray(gens, dtype=np.int32)
    bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
    h = ctypes.c_void_p()
    _check(_lib.ftlm_group_init(gens.shape[1], gens.shape[0], _ptr(gens), bonds.shape[0], _ptr(bonds), float(J),
                                ctypes.byref(h)))
    return Group(h.value)


def ftlm_group_builtin(name: str) -> Group:
    h = ctypes.c_void_p()
    _check(_lib.ftlm_group_builtin(name.encode(), ctypes.byref(h)))
    return Group(h.value)


def ftlm_group_info(g: Group) -> dict:
    n_sites, order, n_irreps = _I(), _I(), _I()
    _check(_lib.ftlm_group_info(g.handle, ctypes.byref(n_sites), ctypes.byref(order), ctypes.byref(n_irreps),
                                None, None, None))
    dims = np.zeros(n_irreps.value, dtype=np.int32)
    fs = np.zeros(n_irreps.value, dtype=np.int32)
    chars = np.zeros((n_irreps.value, order.value))
    _check(_lib.ftlm_group_info(g.handle, None, None, None, _ptr(dims), _ptr(fs), _ptr(chars)))
    weights = np.zeros(n_irreps.value, dtype=np.int32)
    _check(_lib.ftlm_group_weights(g.handle, _ptr(weights)))
    return dict(n_sites=n_sites.value, order=order.value, dims=dims, fs=fs, chars=chars, weights=weights)


def ftlm_group_irrep(g: Group, irrep: int | None = None):
    info = ftlm_group_info(g)
    perms = np.zeros((info["order"], info["n_sites"]), dtype=np.int32)
    rho = None
    if irrep is not None:
        d = int(info["dims"][irrep])
        rho = np.zeros((info["order"], d, d))
    _check(_lib.ftlm_group_irrep(g.handle, -1 if irrep is None else int(irrep), _ptr(rho), _ptr(perms)))
    return rho, perms


def ftlm_group_bonds(g: Group):
    nb, J = _I(), ctypes.c_double()
    _check(_lib.ftlm_group_bonds(g.handle, ctypes.byref(nb), None, ctypes.byref(J)))
    bonds = np.zeros((nb.value, 2), dtype=np.int32)
    _check(_lib.ftlm_group_bonds(g.handle, None, _ptr(bonds), None))
    return bonds, J.value


def ftlm_group_set_irreps(g: Group, rhos) -> None:
    dims = np.array([r.shape[1] for r in rhos], dtype=np.int32)
    flat = np.ascontiguousarray(np.concatenate([np.ascontiguousarray(r, dtype=np.float64).ravel() for r in rhos]))
    _check(_lib.ftlm_group_set_irreps(g.handle, len(rhos), _ptr(dims), _ptr(flat)))


# ---------------------------------------------------------------- sector / block


class Sector:
    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.ftlm_sector_free(self._h)
            self._h = None


class Basis:
    def __init__(self, handle, mask_words=2):
        self._h = handle
        self.mask_words = mask_words  # 4 on spin-flip sectors (256-bit stabilizer masks)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.ftlm_basis_free(self._h)
            self._h = None


def ftlm_build_sector(g: Group, two_s: int, two_M: int, stream=None) -> Sector:
    h = ctypes.c_void_p()
    _check(_lib.ftlm_build_sector(g.handle, two_s, two_M, _stream(stream), ctypes.byref(h)))
    return Sector(h.value)


def ftlm_build_sector_flip(g: Group, two_s: int, stream=None) -> Sector:
    """M = 0 sector under G x Z_2 (spin flip); irreps 2i -> Gamma_i+, 2i + 1 -> Gamma_i-."""
    h = ctypes.c_void_p()
    _check(_lib.ftlm_build_sector_flip(g.handle, two_s, _stream(stream), ctypes.byref(h)))
    return Sector(h.value)


def ftlm_sector_symmetry(s: Sector) -> dict:
    order, n_ir, flip = _I(), _I(), _I()
    _check(_lib.ftlm_sector_symmetry(s.handle, ctypes.byref(order), ctypes.byref(n_ir), ctypes.byref(flip)))
    return dict(order=order.value, n_irreps=n_ir.value, flip=flip.value)


def ftlm_sector_info(s: Sector) -> dict:
    n, dim, nb = _U64(), _U64(), ctypes.c_size_t()
    _check(_lib.ftlm_sector_info(s.handle, ctypes.byref(n), ctypes.byref(dim), ctypes.byref(nb)))
    return dict(n_reps=n.value, sector_dim=dim.value, device_bytes=nb.value)


def ftlm_sector_export(s: Sector):
    n = ftlm_sector_info(s)["n_reps"]
    labels = np.zeros(n, dtype=np.uint64)
    masks = np.zeros((n, 4 if ftlm_sector_symmetry(s)["flip"] else 2), dtype=np.uint64)
    _check(_lib.ftlm_sector_export(s.handle, _ptr(labels), _ptr(masks)))
    return labels, masks


def ftlm_sector_build_entries(s: Sector, stream=None) -> int:
    """Build the sector's entry table (flips -> target, g*, stabilizer); returns the entry count."""
    n = _U64()
    _check(_lib.ftlm_sector_build_entries(s.handle, _stream(stream), ctypes.byref(n)))
    return n.value


def ftlm_sector_free_entries(s: Sector) -> None:
    _check(_lib.ftlm_sector_free_entries(s.handle))


def ftlm_build_block(s: Sector, irrep: int, stream=None) -> Basis:
    h = ctypes.c_void_p()
    _check(_lib.ftlm_build_block(s.handle, irrep, _stream(stream), ctypes.byref(h)))
    return Basis(h.value, 4 if ftlm_sector_symmetry(s)["flip"] else 2)


def ftlm_build_basis(g: Group, two_s: int, two_M: int, irrep: int, stream=None) -> Basis:
    h = ctypes.c_void_p()
    _check(_lib.ftlm_build_basis(g.handle, two_s, two_M, irrep, _stream(stream), ctypes.byref(h)))
    return Basis(h.value)


def ftlm_basis_info(b: Basis) -> dict:
    n, dim, nb = _U64(), _U64(), ctypes.c_size_t()
    _check(_lib.ftlm_basis_info(b.handle, ctypes.byref(n), ctypes.byref(dim), ctypes.byref(nb)))
    return dict(n_reps=n.value, dim=dim.value, device_bytes=nb.value)


def ftlm_basis_export(b: Basis):
    n = ftlm_basis_info(b)["n_reps"]
    labels = np.zeros(n, dtype=np.uint64)
    masks = np.zeros((n, getattr(b, "mask_words", 2)), dtype=np.uint64)
    ng = np.zeros(n, dtype=np.uint8)
    off = np.zeros(n + 1, dtype=np.uint64)
    _check(_lib.ftlm_basis_export(b.handle, _ptr(labels), _ptr(masks), _ptr(ng), _ptr(off)))
    return labels, masks, ng, off


def ftlm_basis_check(b: Basis, stream=None) -> None:
    _check(_lib.ftlm_basis_check(b.handle, _stream(stream)))


class MultiBlock:
    def __init__(self, handle, sector):
        self._h = handle
        self._sector = sector

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.ftlm_multiblock_free(self._h)
            self._h = None


class _Borrowed:
    def __init__(self, handle, owner):
        self.handle = handle
        self._owner = owner


def ftlm_build_multiblock(s: Sector, irreps, stream=None) -> MultiBlock:
    ir = np.ascontiguousarray(irreps, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib.ftlm_build_multiblock(s.handle, len(ir), _ptr(ir), _stream(stream), ctypes.byref(h)))
    return MultiBlock(h.value, s)


def ftlm_multiblock_info(mb: MultiBlock) -> dict:
    n = _I()
    _check(_lib.ftlm_multiblock_info(mb.handle, ctypes.byref(n), None, None))
    dims = np.zeros(n.value, dtype=np.uint64)
    nb = ctypes.c_size_t()
    _check(_lib.ftlm_multiblock_info(mb.handle, None, _ptr(dims), ctypes.byref(nb)))
    return dict(n_blocks=n.value, dims=[int(d) for d in dims], device_bytes=nb.value)


def ftlm_multiblock_block(mb: MultiBlock, k: int):
    h = ctypes.c_void_p()
    _check(_lib.ftlm_multiblock_block(mb.handle, k, ctypes.byref(h)))
    return _Borrowed(h.value, mb)


def ftlm_hv_multi(mb: MultiBlock, dtype: int, B: int, xs, ys, stream=None) -> None:
    n = len(xs)
    dims = ftlm_multiblock_info(mb)["dims"]
    if len(ys) != n or n != len(dims):
        raise ValueError(f"{len(dims)} blocks, got {n} inputs and {len(ys)} outputs")
    xa = (ctypes.c_void_p * n)(*[_dev(x, _vt(dtype), d * B, f"x[{k}]") for k, (x, d) in enumerate(zip(xs, dims))])
    ya = (ctypes.c_void_p * n)(*[_dev(y, _vt(dtype), d * B, f"y[{k}]") for k, (y, d) in enumerate(zip(ys, dims))])
    _check(_lib.ftlm_hv_multi(mb.handle, dtype, B, xa, ya, _stream(stream)))


def ftlm_multiblock_packed_rows(mb: MultiBlock) -> int:
    r = _U64()
    _check(_lib.ftlm_multiblock_packed_rows(mb.handle, ctypes.byref(r)))
    return r.value


def _block_ptrs(mb, dtype, B, blocks):
    dims = ftlm_multiblock_info(mb)["dims"]
    if len(blocks) != len(dims):
        raise ValueError(f"{len(dims)} blocks, got {len(blocks)} arrays")
    n = len(blocks)
    return (ctypes.c_void_p * n)(*[_dev(x, _vt(dtype), d * B, f"block[{k}]")
                                   for k, (x, d) in enumerate(zip(blocks, dims))])


def ftlm_multiblock_pack(mb: MultiBlock, dtype: int, B: int, blocks, packed, stream=None) -> None:
    arr = _block_ptrs(mb, dtype, B, blocks)
    rows = ftlm_multiblock_packed_rows(mb)
    _check(_lib.ftlm_multiblock_pack(mb.handle, dtype, B, arr, _dev(packed, _vt(dtype), rows * B, "packed"),
                                     _stream(stream)))


def ftlm_multiblock_unpack(mb: MultiBlock, dtype: int, B: int, packed, blocks, stream=None) -> None:
    arr = _block_ptrs(mb, dtype, B, blocks)
    rows = ftlm_multiblock_packed_rows(mb)
    _check(_lib.ftlm_multiblock_unpack(mb.handle, dtype, B, _dev(packed, _vt(dtype), rows * B, "packed"), arr,
                                       _stream(stream)))


def ftlm_hv_packed(mb: MultiBlock, dtype: int, B: int, x, y, stream=None) -> None:
    n = ftlm_multiblock_packed_rows(mb) * B
    _check(_lib.ftlm_hv_packed(mb.handle, dtype, B, _dev(x, _vt(dtype), n, "x"), _dev(y, _vt(dtype), n, "y"),
                               _stream(stream)))


def ftlm_fill_label_keyed(b, dtype: int, B: int, seed: int, x, stream=None) -> None:
    """x: device [dim][B] of the dtype; see include/ftlm.h for the definition of the entries."""
    n = ftlm_basis_info(b)["dim"] * B
    _check(_lib.ftlm_fill_label_keyed(b.handle, dtype, B, seed, _dev(x, _vt(dtype), n, "x"), _stream(stream)))


def ftlm_basis_rows(b, labels, stream=None):
    """Packed labels -> (first block row or -1, n_Gamma) per label."""
    lab = np.ascontiguousarray(labels, dtype=np.uint64)
    first = np.zeros(len(lab), dtype=np.int64)
    nrows = np.zeros(len(lab), dtype=np.int32)
    _check(_lib.ftlm_basis_rows(b.handle, len(lab), _ptr(lab), _ptr(first), _ptr(nrows), _stream(stream)))
    return first, nrows


def ftlm_set_autotune(on: int) -> None:
    _check(_lib.ftlm_set_autotune(int(on)))


def ftlm_autotune_report() -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(_lib.ftlm_autotune_report(buf, len(buf)))
    return buf.value.decode()


def ftlm_set_wait_limit(cycles: int) -> None:
    _check(_lib.ftlm_set_wait_limit(int(cycles)))


def ftlm_lanczos_multi(mb: MultiBlock, dtype: int, R: int, n_steps: int, seed: int, block_ids, rng: int = GAUSS,
                       stream=None):
    K = ftlm_multiblock_info(mb)["n_blocks"]
    ids = np.ascontiguousarray(block_ids, dtype=np.uint64)
    alpha = np.zeros((K, R, n_steps))
    beta = np.zeros((K, R, n_steps))
    steps = np.zeros((K, R), dtype=np.int32)
    _check(_lib.ftlm_lanczos_multi(mb.handle, dtype, R, n_steps, seed, _ptr(ids), rng, _stream(stream), _ptr(alpha),
                                   _ptr(beta), _ptr(steps)))
    return alpha, beta, steps


def ftlm_lanczos_sets(sets, dtype: int, R: int, n_steps: int, seed: int, block_ids, rng: int = GAUSS, stream=None):
    """sets: list of MultiBlock with packed layouts; block_ids: [n_sets][K].  Returns alpha, beta
    [n_sets][K][R][n_steps] and steps [n_sets][K][R]."""
    n = len(sets)
    K = ftlm_multiblock_info(sets[0])["n_blocks"]
    arr = (ctypes.c_void_p * n)(*[m.handle for m in sets])
    ids = np.ascontiguousarray(block_ids, dtype=np.uint64).reshape(n, K)
    alpha = np.zeros((n, K, R, n_steps))
    beta = np.zeros((n, K, R, n_steps))
    steps = np.zeros((n, K, R), dtype=np.int32)
    _check(_lib.ftlm_lanczos_sets(n, arr, dtype, R, n_steps, seed, _ptr(ids), rng, _stream(stream), _ptr(alpha),
                                  _ptr(beta), _ptr(steps)))
    return alpha, beta, steps


# ---------------------------------------------------------------- H·v, Lanczos, thermo


def ftlm_hv(b: Basis, dtype: int, B: int, x, y, stream=None) -> None:
    """x, y: device pointers (int) or CUDA tensors of shape [dim, B] (float64 for F64, float32 for F32)."""
    n = ftlm_basis_info(b)["dim"] * B
    _check(_lib.ftlm_hv(b.handle, dtype, B, _dev(x, _vt(dtype), n, "x"), _dev(y, _vt(dtype), n, "y"),
                        _stream(stream)))


def ftlm_lanczos(b: Basis, dtype: int, R: int, n_steps: int, seed: int, block_id: int, rng: int = GAUSS,
                 stream=None):
    alpha = np.zeros((R, n_steps))
    beta = np.zeros((R, n_steps))
    steps = np.zeros(R, dtype=np.int32)
    _check(_lib.ftlm_lanczos(b.handle, dtype, R, n_steps, seed, block_id, rng, _stream(stream), _ptr(alpha),
                             _ptr(beta), _ptr(steps)))
    return alpha, beta, steps


def ftlm_ritz(alpha, beta, steps, stream=None):
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    steps = np.ascontiguousarray(steps, dtype=np.int32)
    n, ld = alpha.shape
    theta = np.zeros((n, ld))
    w = np.zeros((n, ld))
    _check(_lib.ftlm_ritz(n, ld, _ptr(steps), _ptr(alpha), _ptr(beta), _ptr(theta), _ptr(w), _stream(stream)))
    return theta, w


def ftlm_thermo(blocks, T, g=1.0, stream=None):
    """blocks: list of dicts {two_M, d_gamma, dim, alpha[R][ld], beta[R][ld], steps[R]}."""
    keep = []
    arr = (ftlm_block * len(blocks))()
    for i, bl in enumerate(blocks):
        a = np.ascontiguousarray(bl["alpha"], dtype=np.float64)
        be = np.ascontiguousarray(bl["beta"], dtype=np.float64)
        st = np.ascontiguousarray(bl["steps"], dtype=np.int32)
        keep += [a, be, st]
        arr[i] = ftlm_block(int(bl["two_M"]), int(bl["d_gamma"]), int(bl["dim"]), a.shape[0], a.shape[1],
                            _ptr(st), _ptr(a), _ptr(be))
    T = np.ascontiguousarray(T, dtype=np.float64)
    out = [np.zeros(len(T)) for _ in range(4)]
    E0 = np.zeros(1)
    _check(_lib.ftlm_thermo(len(blocks), arr, len(T), _ptr(T), float(g), *[_ptr(o) for o in out], _ptr(E0),
                            _stream(stream)))
    return out[0], out[1], out[2], out[3], float(E0[0])


def ftlm_thermo_noalloc(n_chains, ld, m, alpha, beta, weight, msq, n_T, T, g, out, E0, stream=None) -> None:
    """All array arguments are device addresses (ints) or CUDA tensors; see include/ftlm.h.  n_chains = 0 with
    every array None only makes the library's fixed scratch resident on the current device."""
    nc, nt = int(n_chains), int(n_T)
    f = "float64"
    _check(_lib.ftlm_thermo_noalloc(nc, int(ld), _dev(m, "int32", nc, "m"), _dev(alpha, f, nc * ld, "alpha"),
                                    _dev(beta, f, nc * ld, "beta"), _dev(weight, f, nc, "weight"),
                                    _dev(msq, f, nc, "msq"), nt, _dev(T, f, nt, "T"), float(g),
                                    _dev(out, f, 4 * nt, "out"), _dev(E0, f, 1, "E0"), _stream(stream)))


# ---------------------------------------------------------------- serving loop


class Server:
    """Serving loop (include/ftlm.h): submit jobs, wait for their alpha/beta.  Keeps the groups of
    submitted jobs alive until the server is freed."""

    def __init__(self, cap_bytes: int, n_workers: int = 2, max_parts: int = 64):
        h = ctypes.c_void_p()
        _check(_lib.ftlm_server_create(int(cap_bytes), int(n_workers), int(max_parts), ctypes.byref(h)))
        self._h = h.value
        self._groups = {}
        self._shape = {}

    def submit(self, group: Group, two_s: int, two_M: int, irrep: int, R: int, n_steps: int, seed: int,
               block_id: int, rng: int = GAUSS, dtype: int = F32) -> int:
        j = ftlm_job(group.handle, two_s, two_M, irrep, R, n_steps, seed, block_id, rng, dtype)
        jid = _U64()
        _check(_lib.ftlm_server_submit(self._h, ctypes.byref(j), ctypes.byref(jid)))
        self._groups[id(group)] = group
        self._shape[jid.value] = (R, n_steps)
        return jid.value

    def wait(self, job_id: int, timeout_s: float = -1.0):
        """Returns (info dict, alpha [R][n_steps], beta, steps [R]); raises FtlmError with the job's status."""
        R, n = self._shape[job_id]
        info = ftlm_job_info()
        alpha = np.zeros((R, n))
        beta = np.zeros((R, n))
        steps = np.zeros(R, dtype=np.int32)
        st = _lib.ftlm_server_wait(self._h, job_id, float(timeout_s), ctypes.byref(info), _ptr(alpha), _ptr(beta),
                                   _ptr(steps))
        if st != ETIMEOUT:
            self._shape.pop(job_id, None)
        _check(st)
        return ({f: getattr(info, f) for f, _ in ftlm_job_info._fields_}, alpha, beta, steps)

    def stats(self) -> dict:
        s = ftlm_server_stats()
        _check(_lib.ftlm_server_stats_get(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ftlm_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib.ftlm_server_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


# ---------------------------------------------------------------- profiling

PEAK_LOP3, PEAK_MIN_U32, PEAK_ADD_U64, PEAK_FFMA32, PEAK_DFMA64, PEAK_LDS32, PEAK_GATHER, PEAK_STREAM = range(8)


def ftlm_peak_probe(kind: int, span: int = 0, seg: int = 0, stream=None) -> float:
    """Measured rate of one probe (lane-ops/s, FMAs/s, loads/s or bytes/s; see include/ftlm.h)."""
    r = ctypes.c_double()
    _check(_lib.ftlm_peak_probe(int(kind), int(span), int(seg), _stream(stream), ctypes.byref(r)))
    return r.value



def ftlm_profile_enable(on: bool = True) -> None:
    _check(_lib.ftlm_profile_enable(1 if on else 0))


def ftlm_profile_reset() -> None:
    _check(_lib.ftlm_profile_reset())


def ftlm_profile_get() -> dict:
    p = ftlm_profile()
    _check(_lib.ftlm_profile_get(ctypes.byref(p)))
    return dict(kernel_launches=p.kernel_launches, hv_launches=p.hv_launches, hv_ms=p.hv_ms, hv_rows=p.hv_rows,
                hv_flips=p.hv_flips)
