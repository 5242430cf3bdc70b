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
constants have the central characters as common eigenvectors).  The irreps are
then taken over the reals (Section 3 keeps real arithmetic for irreps of real
Frobenius-Schur type; the real form here extends that to the other two types):

* real type (indicator +1): the irrep itself, chi_R = chi;
* complex type (indicator 0): one entry for the pair Gamma, conj(Gamma), the real
  representation of dimension 2 d_Gamma with chi_R = chi + conj(chi);
* quaternionic type (indicator -1): the real representation of dimension
  2 d_Gamma with chi_R = 2 chi.

Each is realised as an orthogonal representation by projecting the left regular
representation onto its real isotypic component and splitting that with a
random symmetric element of the right-regular commutant.  kappa = <chi_R, chi_R>
(1, 2, 4) is the dimension of the real commutant; a single-partner-row block of
the real form counts every level kappa times its multiplicity in one complex
irrep copy, so its FTLM weight (Eq. 5's d_Gamma) is dim / kappa.
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


KAPPA = {1: 1, 0: 2, -1: 4}  # Frobenius-Schur indicator -> <chi_R, chi_R>


@dataclasses.dataclass
class Irrep:
    dim: int  # dimension of the real representation
    fs: int  # Frobenius-Schur indicator of its complex constituent
    chars: np.ndarray  # [G], chi_R
    rho: np.ndarray | None  # [G, d, d] real orthogonal

    @property
    def kappa(self) -> int:
        return KAPPA[self.fs]

    @property
    def weight(self) -> int:
        """The block's multiplicity factor in Eqs. 5, 6 and 14 (d_Gamma for real type)."""
        return self.dim // self.kappa


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
        # Frobenius-Schur indicator (1/|G|) sum_g chi(g^2), by classes
        sq = np.array([self.class_of[self.mult[c[0], c[0]]] for c in self.classes])
        real_forms, fss, used = [], [], set()
        for t in range(K):
            if t in used:
                continue
            chi = chars[t]
            nu = float(np.real(np.sum(size * chi[sq])) / G)
            fs = int(round(nu))
            if abs(nu - fs) > 1e-6 or fs not in KAPPA:
                raise ArithmeticError("Frobenius-Schur indicator is not 1, 0 or -1")
            if fs == 0:
                conj = [u for u in range(K) if u != t and u not in used
                        and np.max(np.abs(chars[u] - np.conj(chi))) < 1e-8]
                if len(conj) != 1:
                    raise ArithmeticError("complex character without its conjugate")
                used.add(conj[0])
                real_forms.append(2.0 * chi.real)
            elif np.max(np.abs(chi.imag)) > 1e-8:
                raise ArithmeticError("character of real or quaternionic type is not real")
            else:
                real_forms.append((1.0 if fs == 1 else 2.0) * chi.real)
            used.add(t)
            fss.append(fs)
        chars = np.array(real_forms)
        self.class_chars = chars  # [n_irreps, K], chi_R by class
        self.char_table = chars[:, self.class_of]  # [n_irreps, G]
        self._fs = fss

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
        for chi, fs in zip(self.char_table, self._fs):
            d = int(round(chi[0]))
            kappa = KAPPA[fs]
            # real isotypic projector E[x, y] = (d / (kappa |G|)) chi_R(x y^{-1}), rank d^2 / kappa
            E = (d / (kappa * G)) * chi[self.mult[np.arange(G)[:, None], self.inv[None, :]]]
            ev, U = np.linalg.eigh(E)
            W = U[:, ev > 0.5]
            if W.shape[1] * kappa != d * d:
                raise RuntimeError("isotypic component has the wrong dimension")
            # the commutant acts on W as a symmetric matrix over R, C or H: every eigenvalue
            # of a generic one has multiplicity d (one copy of the real irreducible)
            lam, Q = np.linalg.eigh(W.T @ S @ W)
            tol = 1 + abs(lam).max()
            if d > 1 and lam[d - 1] - lam[0] > 1e-8 * tol:
                raise RuntimeError("commutant split did not isolate one irreducible copy")
            if W.shape[1] > d and lam[d] - lam[d - 1] < 1e-6 * tol:
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
            r = ir.rho
            prod = np.einsum("gab,hbc->ghac", r, r)
            res["hom"] = max(res["hom"], float(np.max(np.abs(prod - r[self.mult]))))
            res["orth"] = max(res["orth"], float(np.max(np.abs(
                np.einsum("gab,gcb->gac", r, r) - np.eye(ir.dim)[None]))))
            res["char"] = max(res["char"], float(np.max(np.abs(np.trace(r, axis1=1, axis2=2) - ir.chars))))
        ct = self.char_table
        kap = np.diag([ir.kappa for ir in self.irreps])
        res["row_orth"] = float(np.max(np.abs(ct @ ct.T / G - kap)))
        # sum over the complex irreps of d^2: a complex pair gives 2 (d/2)^2, a quaternionic one (d/2)^2
        res["sum_d2"] = int(sum(ir.dim ** 2 // ir.kappa for ir in self.irreps))
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
                rho = np.concatenate([ir.rho, sgn * ir.rho])
                self.irreps.append(Irrep(ir.dim, ir.fs, np.concatenate([ir.chars, sgn * ir.chars]), rho))
        self.char_table = np.array([ir.chars for ir in self.irreps])
