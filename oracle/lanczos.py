"""Oracle FTLM driver: start vectors, Lanczos, Ritz pairs, thermal sums.

* Start vectors (Section 2.2: real normalised Gaussian per block).  Random bits
  come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), implemented here
  from its published definition: key (k0, k1) = (low 32 bits of seed, low 32
  bits of block_id); counter (c0, c1, c2, c3) = (low and high 32 bits of the
  row index, chain index, 0).  Gaussian: Box-Muller in FP64 with
  U1 = (((x0 >> 5) << 26 | x1 >> 6) + 0.5) 2^-53 and
  U2 = ((x2 >> 5) << 26 | x3 >> 6) 2^-53, z = sqrt(-2 ln U1) cos(2 pi U2).
  Rademacher: z = +1 if x0 is even, else -1.  Each chain is normalised in FP64.
* Lanczos (Section 2.2): w = H v_j; alpha_j = <v_j, w>; w -= alpha_j v_j +
  beta_j v_{j-1}; beta_{j+1} = |w|; v_{j+1} = w / beta_{j+1}.  A chain stops
  after step j when beta_{j+1} <= 1e-12 (|alpha_j| + beta_j) or j + 1 reaches
  min(N_L, dim).  beta[j] stores beta_{j+1}.
* Ritz pairs: eigenvalues theta_k of the tridiagonal matrix and weights
  w_k = (first eigenvector component)^2 (Section 2.2), via LAPACK.
* Thermal sums (Eqs. 5-7 with the weights of Eq. 14): every chain of block
  (M, Gamma) carries W = mult_M d_Gamma D_{M,Gamma} / R; all exponentials are
  shifted by the global E0 = min theta; C = beta^2 <(H - <H>)^2>;
  chi = g^2 beta sum mult_M M^2 Z_M / sum mult_M Z_M; ln Z reported.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

MASK = np.uint64(0xFFFFFFFF)
M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 values held in uint64 arrays."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def start_vectors(dim, R, seed, block_id, rng="gauss", chain0=0):
    """[dim, R] normalised start vectors, chains chain0 .. chain0+R-1."""
    rows = np.arange(dim, dtype=np.uint64)
    out = np.empty((dim, R))
    for r in range(R):
        x0, x1, x2, x3 = philox4x32_10(rows & MASK, rows >> np.uint64(32), np.uint64(chain0 + r), 0, seed, block_id)
        if rng == "gauss":
            u1 = (((x0 >> np.uint64(5)) << np.uint64(26)) | (x1 >> np.uint64(6))).astype(np.float64)
            u1 = (u1 + 0.5) * 2.0 ** -53
            u2 = (((x2 >> np.uint64(5)) << np.uint64(26)) | (x3 >> np.uint64(6))).astype(np.float64) * 2.0 ** -53
            z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        elif rng == "rademacher":
            z = np.where((x0 & np.uint64(1)) == 0, 1.0, -1.0)
        else:
            raise ValueError(rng)
        out[:, r] = z / np.sqrt(np.sum(z * z))
    return out


def lanczos(hv, v0, n_steps, tol=1e-12):
    """One chain: returns (alpha[m], beta[m]) with beta[j] = beta_{j+1}."""
    dim = v0.shape[0]
    m_max = min(n_steps, dim)
    alpha, beta = [], []
    v_prev = np.zeros_like(v0)
    v = v0.copy()
    b = 0.0
    for j in range(m_max):
        w = hv(v)
        a = float(v @ w)
        w = w - a * v - b * v_prev
        bn = float(np.sqrt(w @ w))
        alpha.append(a)
        beta.append(bn)
        if j + 1 == m_max or bn <= tol * (abs(a) + b):
            break
        v_prev, v, b = v, w / bn, bn
    return np.array(alpha), np.array(beta)


def ritz(alpha, beta):
    m = len(alpha)
    if m == 1:
        return np.array(alpha, dtype=float), np.ones(1)
    theta, Z = scipy.linalg.eigh_tridiagonal(np.asarray(alpha), np.asarray(beta[: m - 1]))
    return theta, Z[0, :] ** 2


def thermo(blocks, T, g=1.0):
    """blocks: list of dicts {two_M, d_gamma, dim, R, alpha: [R][m], beta: [R][m]} (ragged m allowed).

    Returns lnZ, E, C, chi (arrays over T) and E0.
    """
    entries = []  # (theta, weight, M^2, M-key)
    for blk in blocks:
        mult = 2.0 if blk["two_M"] > 0 else 1.0
        Wc = mult * blk["d_gamma"] * blk["dim"] / blk["R"]
        Msq = (blk["two_M"] / 2.0) ** 2
        for a, b in zip(blk["alpha"], blk["beta"]):
            th, w = ritz(a, b)
            entries.append((th, Wc * w, Msq))
    theta = np.concatenate([e[0] for e in entries])
    W = np.concatenate([e[1] for e in entries])
    Msq = np.concatenate([np.full(len(e[0]), e[2]) for e in entries])
    E0 = float(theta.min())
    T = np.asarray(T, dtype=float)
    lnZ, E, C, chi = (np.empty(len(T)) for _ in range(4))
    for t, temp in enumerate(T):
        beta = 1.0 / temp
        boltz = W * np.exp(-beta * (theta - E0))
        Z = boltz.sum()
        Em = (boltz * theta).sum() / Z
        C[t] = beta * beta * (boltz * (theta - Em) ** 2).sum() / Z
        E[t] = Em
        lnZ[t] = np.log(Z) - beta * E0
        chi[t] = g * g * beta * (boltz * Msq).sum() / Z
    return lnZ, E, C, chi, E0
