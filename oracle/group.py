"""Oracle group module: closure, classes, characters and real irreps (Section 3).

Conventions (shared with the library only as documented conventions, not code):

* A group element g is its site permutation ``perm[k] = pi_g(k)``.  It acts on a
  product state by moving the digit of site k to site pi_g(k), so that
  U(g)U(h) = U(gh) with pi_gh = pi_g o pi_h.
* Canonical element order: lexicographic order of the arrays
  (pi_g(0), ..., pi_g(N-1)); the identity is first.
* Canonical irrep order: dimension ascending, then the character vector (over
  the canonical element order, rounded to 1e-8) lexicographically descending,
  so the trivial irrep is first.

The character table comes from the class algebra (the class-sum structure
constants have the central characters as common eigenvectors); every irrep of
real Frobenius-Schur type is then realised as an orthogonal representation by
projecting the left regular representation onto its isotypic component and
splitting that with a random symmetric element of the right-regular commutant.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def compose(p, q):
    """pi_{pq} = pi_p o pi_q."""
    return tuple(p[k] for k in q)


def close_group(gens, max_order=100000):
    """All products of the generators (breadth-first closure), canonical order."""
    gens = [tuple(int(v) for v in g) for g in gens]
    n = len(gens[0]) if gens else 0
    for g in gens:
        if sorted(g) != list(range(n)):
            raise ValueError("generator is not a permutation")
    ident = tuple(range(n))
    seen = {ident}
    frontier = [ident]
    while frontier:
        nxt = []
        for a in frontier:
            for g in gens:
                c = compose(g, a)
                if c not in seen:
                    seen.add(c)
                    nxt.append(c)
                    if len(seen) > max_order:
                        raise ValueError("group larger than max_order")
        frontier = nxt
    return np.array(sorted(seen), dtype=np.int32)


@dataclasses.dataclass
class Irrep:
    dim: int
    fs: int  # Frobenius-Schur indicator
    chars: np.ndarray  # [G]
    rho: np.ndarray | None  # [G, d, d] real orthogonal, None if not of real type


class Group:
    """A finite permutation group with its real irreps."""

    def __init__(self, gens, bonds=None, seed=12345):
        self.perms = close_group(gens)
        self.order = G = len(self.perms)
        self.n_sites = self.perms.shape[1]
        index = {tuple(p): i for i, p in enumerate(self.perms.tolist())}
        self.index = index
        self.mult = np.empty((G, G), dtype=np.int64)
        for i, p in enumerate(self.perms.tolist()):
            for j, q in enumerate(self.perms.tolist()):
                self.mult[i, j] = index[compose(p, q)]
        self.inv = np.array([int(np.nonzero(self.mult[i] == 0)[0][0]) for i in range(G)])
        if bonds is not None:
            self.check_bonds(bonds)
        self._classes()
        self._character_table(seed)
        self._irreps(seed)

    def check_bonds(self, bonds):
        bs = {tuple(sorted((int(i), int(j)))) for i, j in bonds}
        for p in self.perms:
            img = {tuple(sorted((int(p[i]), int(p[j])))) for i, j in bs}
            if img != bs:
                raise ValueError("bond list is not invariant under the group")

    # ---- conjugacy classes -------------------------------------------------
    def _classes(self):
        G = self.order
        cls = -np.ones(G, dtype=np.int64)
        classes = []
        for g in range(G):
            if cls[g] >= 0:
                continue
            members = sorted({int(self.mult[self.mult[h, g], self.inv[h]]) for h in range(G)})
            for m in members:
                cls[m] = len(classes)
            classes.append(members)
        self.classes = classes
        self.class_of = cls

    # ---- character table from the class algebra ---------------------------
    def _character_table(self, seed):
        G, K = self.order, len(self.classes)
        size = np.array([len(c) for c in self.classes], dtype=float)
        # a[i, j, k] = #{x in C_i : x^{-1} z_k in C_j}, z_k the first element of C_k
        a = np.zeros((K, K, K))
        for k in range(K):
            z = self.classes[k][0]
            for i in range(K):
                for x in self.classes[i]:
                    a[i, self.class_of[self.mult[self.inv[x], z]], k] += 1
        rng = np.random.default_rng(seed)
        c = rng.standard_normal(K)
        A = np.einsum("i,ijk->jk", c, a)
        _, vecs = np.linalg.eig(A)
        chars = []
        e_cls = int(self.class_of[0])
        for t in range(K):
            w = vecs[:, t] / vecs[e_cls, t]
            d = np.sqrt(G / np.sum(np.abs(w) ** 2 / size))
            chi_cls = d * w / size
            chars.append(chi_cls)
        chars = np.array(chars)
        if np.max(np.abs(chars.imag)) > 1e-8:
            raise NotImplementedError("complex characters are outside the oracle's real path")
        chars = chars.real
        self.class_chars = chars  # [n_irreps, K]
        self.char_table = chars[:, self.class_of]  # [n_irreps, G]

    # ---- real irreps ------------------------------------------------------
    def _regular(self, g):
        """L(g) e_y = e_{g y} as a permutation array: image index of each basis vector."""
        return self.mult[g]

    def _irreps(self, seed):
        G = self.order
        rng = np.random.default_rng(seed + 1)
        # random symmetric element of the commutant of L: S = sum_h c_h (R(h) + R(h)^T),
        # R(h) e_y = e_{y h^{-1}}; S[x, y] = c[x^{-1} y] + c[y^{-1} x]
        cvec = rng.standard_normal(G)
        X = self.mult[self.inv][:, :]  # X[x, y] = x^{-1} y
        S = cvec[X] + cvec[X.T]
        irreps = []
        for chi in self.char_table:
            d = int(round(chi[0]))
            fs = int(round(np.sum(chi[self.mult[np.arange(G), np.arange(G)]]) / G))
            if fs != 1:
                irreps.append(Irrep(d, fs, chi.copy(), None))
                continue
            # isotypic projector E[x, y] = (d/|G|) chi(x y^{-1})
            E = (d / G) * chi[self.mult[np.arange(G)[:, None], self.inv[None, :]]]
            ev, U = np.linalg.eigh(E)
            W = U[:, ev > 0.5]
            if W.shape[1] != d * d:
                raise RuntimeError("isotypic component has the wrong dimension")
            lam, Q = np.linalg.eigh(W.T @ S @ W)
            if d > 1 and not (lam[d - 1] - lam[0] < 1e-8 * (1 + abs(lam).max())
                              and lam[d] - lam[d - 1] > 1e-6 * (1 + abs(lam).max())):
                raise RuntimeError("commutant split did not isolate one irreducible copy")
            Bm = W @ Q[:, :d]
            rho = np.empty((G, d, d))
            for g in range(G):
                # (L(g) B)[y] = B[g^{-1} y]
                rho[g] = Bm.T @ Bm[self.mult[self.inv[g]]]
            irreps.append(Irrep(d, fs, chi.copy(), rho))
        key = [(ir.dim, tuple(-np.round(ir.chars, 8))) for ir in irreps]
        order = sorted(range(len(irreps)), key=lambda i: key[i])
        self.irreps = [irreps[i] for i in order]
        self.char_table = np.array([ir.chars for ir in self.irreps])

    # ---- checks -----------------------------------------------------------
    def verify_irreps(self, tol=1e-10):
        """Max residuals of homomorphism, orthogonality and character identities."""
        G = self.order
        res = {"hom": 0.0, "orth": 0.0, "char": 0.0}
        for ir in self.irreps:
            if ir.rho is None:
                continue
            r = ir.rho
            prod = np.einsum("gab,hbc->ghac", r, r)
            res["hom"] = max(res["hom"], float(np.max(np.abs(prod - r[self.mult]))))
            res["orth"] = max(res["orth"], float(np.max(np.abs(
                np.einsum("gab,gcb->gac", r, r) - np.eye(ir.dim)[None]))))
            res["char"] = max(res["char"], float(np.max(np.abs(np.trace(r, axis1=1, axis2=2) - ir.chars))))
        ct = self.char_table
        res["row_orth"] = float(np.max(np.abs(ct @ ct.T / G - np.eye(len(ct)))))
        res["sum_d2"] = int(sum(ir.dim ** 2 for ir in self.irreps))
        return res

    def element(self, perm):
        return self.index[tuple(int(v) for v in perm)]


class SpinFlipExtended:
    """G x Z_2 at M = 0 (Section 2.2): the global spin flip m -> -m commutes with H and with
    every site permutation.  Element (g, z) has canonical index g + z |G| (z = 1 after all of
    G) and is stored as the signed permutation pi_g(k) + z N: the digit of site k moves to
    pi_g(k) as a_k (z = 0) or as 2s - a_k (z = 1).  Each real irrep Gamma of G gives
    Gamma+ (rho(g, z) = rho(g)) and Gamma- (rho(g, z) = (-1)^z rho(g)); in the canonical irrep
    order (dimension, then characters descending) they are interleaved: 2i -> Gamma_i+,
    2i + 1 -> Gamma_i-."""

    def __init__(self, group):
        self.base = group
        G, N = group.order, group.n_sites
        self.order = 2 * G
        self.n_sites = N
        self.perms = np.concatenate([group.perms, group.perms + N]).astype(np.int32)
        self.inv = np.concatenate([group.inv, group.inv + G])
        self.mult = np.empty((2 * G, 2 * G), dtype=np.int64)
        for z in (0, 1):
            for w in (0, 1):
                self.mult[z * G:(z + 1) * G, w * G:(w + 1) * G] = group.mult + ((z ^ w) * G)
        self.classes = [list(c) for c in group.classes] + [[g + G for g in c] for c in group.classes]
        self.irreps = []
        for ir in group.irreps:
            for sgn in (1.0, -1.0):
                rho = None if ir.rho is None else np.concatenate([ir.rho, sgn * ir.rho])
                self.irreps.append(Irrep(ir.dim, ir.fs, np.concatenate([ir.chars, sgn * ir.chars]), rho))
        self.char_table = np.array([ir.chars for ir in self.irreps])
