"""Build and load the C part of the oracle (``ftlm_oracle.c``) via ctypes."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ftlm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (OpenMP) if it is missing or stale."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"])
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        L.or_enumerate.restype = ctypes.c_int64
        L.or_enumerate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int64]
        L.or_min_rep.restype = ctypes.c_int
        L.or_min_rep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_uint64, P, P]
        L.or_hv_rows.restype = ctypes.c_int
        L.or_hv_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P,
                                 ctypes.c_double, ctypes.c_int64, P, P, P, P, P, P, ctypes.c_int, P, ctypes.c_int,
                                 P, P, P, ctypes.c_int64]
        L.or_stab.restype = ctypes.c_int
        L.or_stab.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_uint64, P]
        L.or_flip_entries.restype = ctypes.c_int
        L.or_flip_entries.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_int, P, P, P, P]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def enumerate_reps(n_sites, d, A, perms):
    """Sorted orbit representatives and stabilizer bitmasks (uint64 words) of one sector."""
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    G = perms.shape[0]
    W = (G + 63) // 64
    cap = 1 << 16
    while True:
        reps = np.empty(cap, dtype=np.uint64)
        stab = np.empty((cap, W), dtype=np.uint64)
        n = lib().or_enumerate(n_sites, d, A, G, ptr(perms), ptr(reps), ptr(stab), cap)
        if n < -(1 << 62):
            raise ValueError("bad arguments to or_enumerate")
        if n >= 0:
            return reps[:n].copy(), stab[:n].copy()
        cap = -n


def min_rep(n_sites, d, perms, label):
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    rep = np.zeros(1, dtype=np.uint64)
    g = np.zeros(1, dtype=np.int32)
    lib().or_min_rep(n_sites, d, perms.shape[0], ptr(perms), int(label), ptr(rep), ptr(g))
    return int(rep[0]), int(g[0])


def stabilizer(n_sites, d, perms, label):
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    G = perms.shape[0]
    mask = np.zeros((G + 63) // 64, dtype=np.uint64)
    lib().or_stab(n_sites, d, G, ptr(perms), int(label), ptr(mask))
    return mask


def flip_entries(n_sites, two_s, perms, bonds, J, label):
    """(r' labels, g*, c_a, diagonal energy) of every off-diagonal term acting on one representative."""
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    bonds = np.ascontiguousarray(bonds, dtype=np.int32)
    cap = 2 * len(bonds)
    rp = np.zeros(cap, dtype=np.uint64)
    gs = np.zeros(cap, dtype=np.int32)
    cf = np.zeros(cap)
    dg = np.zeros(1)
    n = lib().or_flip_entries(n_sites, two_s + 1, two_s, perms.shape[0], ptr(perms), len(bonds), ptr(bonds),
                              float(J), int(label), cap, ptr(rp), ptr(gs), ptr(cf), ptr(dg))
    if n < 0:
        raise RuntimeError("or_flip_entries failed")
    return rp[:n], gs[:n], cf[:n], float(dg[0])


def num_threads() -> int:
    return int(lib().or_num_threads())
