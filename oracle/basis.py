"""Oracle symmetry-adapted basis of one (M, Gamma) block (Section 2.3).

* Representatives: smallest label of each orbit (Section 2.3), brute force in C.
* Stabilizer (Eq. 8): bitmask of the group elements fixing the representative.
* n_Gamma(r) = (1/|Stab|) sum_{h in Stab} chi_Gamma(h)  (rounded, residual checked).
* V_r (Eq. 11): orthonormal basis of the range of the projector
  (1/|Stab|) sum_h rho_Gamma(h), which is (|G|/(d |Stab|)) times the Gram matrix of
  Eq. 10.  The range has no preferred basis; the oracle takes modified
  Gram-Schmidt over the projector's columns in column order, accepting a column
  when its residual norm exceeds 1e-8.  A trivial stabilizer gives V_r = I.
* Row offsets: prefix sum of n_Gamma(r) in label order (Eq. 13 gives the total).
"""
from __future__ import annotations

import numpy as np

from . import native
from .sector import digit_total


class SectorBasis:
    def __init__(self, group, two_s: int, two_M: int):
        self.group = group
        self.two_s, self.two_M = two_s, two_M
        self.n_sites = group.n_sites
        self.d = two_s + 1
        self.A = digit_total(self.n_sites, two_s, two_M)
        self.reps, self.stab = native.enumerate_reps(self.n_sites, self.d, self.A, group.perms)
        keys, inverse = np.unique(self.stab, axis=0, return_inverse=True)
        self.stab_keys = keys
        self.stab_index = inverse.reshape(-1)
        self.stab_elems = [self._elements(k) for k in keys]

    def _elements(self, words):
        G = self.group.order
        return np.array([g for g in range(G) if (int(words[g // 64]) >> (g % 64)) & 1], dtype=np.int64)

    @property
    def n_reps(self) -> int:
        return len(self.reps)


def gram_schmidt_range(P, tol=1e-8):
    """Orthonormal columns spanning range(P): MGS over P's columns in order."""
    d = P.shape[0]
    Q = []
    for j in range(d):
        v = P[:, j].copy()
        for q in Q:
            v -= (q @ v) * q
        nrm = np.linalg.norm(v)
        if nrm > tol:
            Q.append(v / nrm)
    V = np.zeros((d, d))
    for k, q in enumerate(Q):
        V[:, k] = q
    return V, len(Q)


class BlockBasis:
    def __init__(self, sector: SectorBasis, irrep: int):
        self.sector = sector
        g = sector.group
        ir = g.irreps[irrep]
        if ir.rho is None:
            raise NotImplementedError("irrep is not of real type")
        self.irrep = irrep
        self.dG = dG = ir.dim
        self.rho = np.ascontiguousarray(ir.rho)
        ns = len(sector.stab_elems)
        self.stab_n = np.zeros(ns, dtype=np.int32)
        self.stab_V = np.zeros((ns, dG, dG))
        self.stab_sqrt = np.zeros(ns)
        for t, S in enumerate(sector.stab_elems):
            val = float(np.sum(ir.chars[S])) / len(S)
            nG = int(round(val))
            if abs(val - nG) > 1e-6:
                raise ArithmeticError("n_Gamma is not an integer")
            P = ir.rho[S].sum(axis=0) / len(S)
            V, cnt = gram_schmidt_range(P)
            if cnt != nG:
                raise ArithmeticError("projector rank differs from the character count")
            self.stab_n[t], self.stab_V[t], self.stab_sqrt[t] = nG, V, np.sqrt(len(S))
        idx = sector.stab_index
        self.n = self.stab_n[idx].astype(np.int32)
        self.off = np.zeros(sector.n_reps + 1, dtype=np.int64)
        np.cumsum(self.n, out=self.off[1:])
        self.dim = int(self.off[-1])
        self.vidx = idx.astype(np.int64)
        self.sqrtS = self.stab_sqrt[idx]

    def hv(self, x, rows=None):
        """y = H x (x: [dim] or [dim, B]); rows: representative indices to fill (others left 0)."""
        sec, g = self.sector, self.sector.group
        x = np.asarray(x, dtype=np.float64)
        squeeze = x.ndim == 1
        X = np.ascontiguousarray(x.reshape(self.dim, -1))
        B = X.shape[1]
        Y = np.zeros_like(X)
        bonds = np.ascontiguousarray(self.bonds, dtype=np.int32)
        rows_arr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        inv = np.ascontiguousarray(g.inv, dtype=np.int32)
        st = native.lib().or_hv_rows(
            sec.n_sites, sec.d, sec.two_s, g.order, native.ptr(g.perms), native.ptr(inv), len(bonds),
            native.ptr(bonds), float(self.J), sec.n_reps, native.ptr(sec.reps), native.ptr(self.n),
            native.ptr(self.off), native.ptr(self.sqrtS), native.ptr(self.vidx),
            native.ptr(np.ascontiguousarray(self.stab_V)), self.dG, native.ptr(self.rho), B, native.ptr(X),
            native.ptr(Y), native.ptr(rows_arr), 0 if rows_arr is None else len(rows_arr))
        if st != 0:
            raise RuntimeError("flipped state's representative missing from the table")
        return Y.reshape(-1) if squeeze else Y

    # the Hamiltonian (bonds, J) is attached by the caller
    bonds = None
    J = 1.0

    def with_hamiltonian(self, bonds, J=1.0):
        self.bonds = np.asarray(bonds, dtype=np.int32)
        self.J = float(J)
        return self

    def dense(self):
        """Dense block matrix built column by column from hv (small blocks only)."""
        return self.hv(np.eye(self.dim))


def block(group, bonds, two_s, two_M, irrep, J=1.0, sector=None):
    sec = sector if sector is not None else SectorBasis(group, two_s, two_M)
    return BlockBasis(sec, irrep).with_hamiltonian(bonds, J)


def hv_rows_by_label(group, irrep, bonds, J, two_s, rep_labels, xvals):
    """Rows of y = H x for the given representatives, without a representative table.

    rep_labels: base-(2s+1) labels of orbit representatives.  xvals(label, n)
    returns the [n, B] block-vector rows of representative ``label``.  Every
    quantity is computed from the label itself: the off-diagonal terms of the
    representative (flipped label, its orbit minimum r' and g*, c_a of Eq. 3),
    the stabilizers of r and r' (Eq. 8) with their n_Gamma and V (Eqs. 10-11),
    and the pull form of Eq. 15 plus Eq. 16.  Returns a list of [n_Gamma(r), B].
    """
    from . import native

    ir = group.irreps[irrep]
    if ir.rho is None:
        raise NotImplementedError("irrep is not of real type")
    N, d = group.n_sites, two_s + 1
    cache = {}

    def stab_info(label):
        mask = native.stabilizer(N, d, group.perms, label)
        key = tuple(int(w) for w in mask)
        if key not in cache:
            S = np.array([g for g in range(group.order) if (key[g // 64] >> (g % 64)) & 1])
            val = float(np.sum(ir.chars[S])) / len(S)
            nG = int(round(val))
            P = ir.rho[S].sum(axis=0) / len(S)
            V, cnt = gram_schmidt_range(P)
            if cnt != nG:
                raise ArithmeticError("projector rank differs from the character count")
            cache[key] = (nG, V, np.sqrt(len(S)))
        return cache[key]

    out = []
    for r in rep_labels:
        r = int(r)
        n_r, V_r, sq_r = stab_info(r)
        if n_r == 0:
            out.append(None)
            continue
        rp, gs, cf, diag = native.flip_entries(N, two_s, group.perms, bonds, J, r)
        x_r = xvals(r, n_r)
        y = diag * x_r
        for lab, g_star, c in zip(rp.tolist(), gs.tolist(), cf.tolist()):
            n_j, V_j, sq_j = stab_info(lab)
            if n_j == 0:
                continue
            g_e = group.inv[g_star]
            M = V_r.T @ ir.rho[g_e] @ V_j
            y = y + (c * sq_j / sq_r) * (M[:n_r, :n_j] @ xvals(lab, n_j))
        out.append(y)
    return out
