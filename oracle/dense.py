"""Dense references for tiny clusters (Section 4.1's dense projector check).

* ``sector_hamiltonian``: Eq. 1 in the product basis of one M sector, built
  entry by entry from Eq. 3 (off-diagonal) and J m_i m_j (diagonal).
* ``projected_basis``: the explicit symmetry-adapted vectors of Eq. 12 at
  partner row alpha = 1,
      psi_{r,k} = d_Gamma / (|G| sqrt(lambda_r)) sum_g [rho(g)^* V_r]_{1,k} U(g)|r>,
  lambda_r = d_Gamma |Stab r| / |G|, written out in the sector's product basis.
"""
from __future__ import annotations

import math

import numpy as np

from .sector import digit_total


def _digits(n, N, d):
    a = []
    for _ in range(N):
        a.append(n % d)
        n //= d
    return a


def _label(a, d):
    n = 0
    for v in reversed(a):
        n = n * d + v
    return n


def sector_labels(n_sites, two_s, two_M):
    d = two_s + 1
    A = digit_total(n_sites, two_s, two_M)
    return [n for n in range(d ** n_sites) if sum(_digits(n, n_sites, d)) == A]


def sector_hamiltonian(n_sites, two_s, two_M, bonds, J=1.0):
    d = two_s + 1
    s = two_s / 2
    labels = sector_labels(n_sites, two_s, two_M)
    pos = {n: i for i, n in enumerate(labels)}
    H = np.zeros((len(labels), len(labels)))
    for col, n in enumerate(labels):
        a = _digits(n, n_sites, d)
        for i, j in bonds:
            mi, mj = a[i] - s, a[j] - s
            H[col, col] += J * mi * mj
            for sgn in (+1, -1):
                ai, aj = a[i] + sgn, a[j] - sgn
                if not (0 <= ai <= two_s and 0 <= aj <= two_s):
                    continue
                c = 0.5 * J * math.sqrt(s * (s + 1) - mi * (mi + sgn)) * math.sqrt(s * (s + 1) - mj * (mj - sgn))
                b = list(a)
                b[i], b[j] = ai, aj
                H[pos[_label(b, d)], col] += c
    return labels, H


def full_hamiltonian(n_sites, two_s, bonds, J=1.0):
    """Eq. 1 over the whole (2s+1)^N space (every M)."""
    d = two_s + 1
    s = two_s / 2
    D = d ** n_sites
    H = np.zeros((D, D))
    for n in range(D):
        a = _digits(n, n_sites, d)
        for i, j in bonds:
            mi, mj = a[i] - s, a[j] - s
            H[n, n] += J * mi * mj
            for sgn in (+1, -1):
                ai, aj = a[i] + sgn, a[j] - sgn
                if not (0 <= ai <= two_s and 0 <= aj <= two_s):
                    continue
                c = 0.5 * J * math.sqrt(s * (s + 1) - mi * (mi + sgn)) * math.sqrt(s * (s + 1) - mj * (mj - sgn))
                b = list(a)
                b[i], b[j] = ai, aj
                H[_label(b, d), n] += c
    return H


def projected_basis(block, labels):
    """Columns psi_{r,k} (Eq. 12, alpha = 1) in the product basis ``labels``."""
    sec = block.sector
    g = sec.group
    G, dG = g.order, block.dG
    pos = {n: i for i, n in enumerate(labels)}
    Psi = np.zeros((len(labels), block.dim))
    for i, r in enumerate(sec.reps.tolist()):
        nr = int(block.n[i])
        if nr == 0:
            continue
        V = block.stab_V[block.vidx[i]]
        lam = dG * block.sqrtS[i] ** 2 / G
        a = _digits(int(r), sec.n_sites, sec.d)
        for gi in range(G):
            b = [0] * sec.n_sites
            for k, p in enumerate(g.perms[gi]):
                if p < sec.n_sites:
                    b[p] = a[k]
                else:  # element of G x Z_2 with the spin flip: the digit moves as 2s - a_k
                    b[p - sec.n_sites] = sec.d - 1 - a[k]
            row = pos[_label(b, sec.d)]
            coef = (g.irreps[block.irrep].rho[gi] @ V)[0, :nr]  # real irreps: rho^* = rho
            Psi[row, block.off[i]:block.off[i] + nr] += dG / (G * math.sqrt(lam)) * coef
    return Psi
