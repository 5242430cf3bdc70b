"""Sector and block dimensions (Section 2.1, Eq. 13; Table 1 and Table 2 counts).

* ``sector_dim``: number of base-d digit strings of length N (d = 2s+1) whose
  digit sum is A_tot = N s + M (Section 2.1), by the plain counting recursion
  over sites.
* ``fixed_count``: number of M-sector product states left unchanged by one site
  permutation: the digits must be constant on every cycle of the permutation
  (with the spin flip of G x Z_2 at M = 0: alternate between a and 2s - a).
* ``block_dim``: the single-partner-row block dimension of irrep Gamma, i.e. the
  multiplicity of Gamma in the permutation representation on the M sector,
  (1/|G|) sum_g chi_Gamma(g) * fixed_count(g)  (equals Eq. 13 summed over the
  orbits: sum_r n_Gamma(r)).
"""
from __future__ import annotations


def digit_total(n_sites: int, two_s: int, two_M: int) -> int:
    twice = n_sites * two_s + two_M
    if twice % 2:
        raise ValueError("N*s + M is not an integer")
    return twice // 2


def count_strings(lengths, dmax: int, total: int) -> int:
    """Ways to give each cycle (of the given lengths) one digit in 0..dmax, sum(len*digit) = total."""
    ways = [0] * (total + 1)
    ways[0] = 1
    for ell in lengths:
        new = [0] * (total + 1)
        for a, w in enumerate(ways):
            if w == 0:
                continue
            for v in range(dmax + 1):
                t = a + ell * v
                if t > total:
                    break
                new[t] += w
        ways = new
    return ways[total]


def sector_dim(n_sites: int, two_s: int, two_M: int) -> int:
    A = digit_total(n_sites, two_s, two_M)
    if A < 0 or A > n_sites * two_s:
        return 0
    return count_strings([1] * n_sites, two_s, A)


def cycle_lengths(perm) -> list[int]:
    perm = list(perm)
    seen = [False] * len(perm)
    out = []
    for k in range(len(perm)):
        if seen[k]:
            continue
        ell, j = 0, k
        while not seen[j]:
            seen[j] = True
            j = perm[j]
            ell += 1
        out.append(ell)
    return out


def fixed_count(perm, two_s: int, two_M: int) -> int:
    N = len(perm)
    A = digit_total(N, two_s, two_M)
    if A < 0 or A > N * two_s:
        return 0
    if any(p >= N for p in perm):
        # element of G x Z_2 with the spin flip (entries pi(k) + N): a fixed state has
        # a_{pi(k)} = 2s - a_k, so along a cycle the digits alternate a, 2s - a.  An even
        # cycle takes any a (its digit sum is len * s); an odd one needs a = s, possible
        # only for integer s.  Every fixed state then has digit sum N s, i.e. M = 0.
        if two_M != 0:
            return 0
        count = 1
        for ell in cycle_lengths([p % N for p in perm]):
            if ell % 2 == 0:
                count *= two_s + 1
            elif two_s % 2:
                return 0
        return count
    return count_strings(cycle_lengths(perm), two_s, A)


def block_dims(group, two_s: int, two_M: int) -> list[int]:
    """Block dimension of every irrep (canonical irrep order) by the character formula."""
    G = group.order
    fix = {}
    out = []
    for ir in group.irreps:
        tot = 0.0
        for cls in group.classes:
            g = cls[0]
            if g not in fix:
                fix[g] = fixed_count(group.perms[g], two_s, two_M)
            tot += len(cls) * ir.chars[g] * fix[g]
        val = tot / G
        r = int(round(val))
        if abs(val - r) > 1e-3 * max(1.0, abs(val)) ** 0.5:
            raise ArithmeticError(f"character sum not an integer: {val}")
        out.append(r)
    return out
