"""Exact-arithmetic brute force for tiny inputs (test helper, pins the oracle).

Determinants are exact rationals (Python Fraction, every float64 converts
exactly); square roots use the decimal module at 80 significant digits.  This
is pure-Python and only meant for k <= 5 modes.
"""
from __future__ import annotations

from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np

getcontext().prec = 80


def det_exact(A) -> Fraction:
    """Determinant of a square matrix of Fractions by fraction-exact elimination."""
    n = len(A)
    a = [[Fraction(x) for x in row] for row in A]
    det = Fraction(1)
    for j in range(n):
        p = next((i for i in range(j, n) if a[i][j] != 0), None)
        if p is None:
            return Fraction(0)
        if p != j:
            a[j], a[p] = a[p], a[j]
            det = -det
        det *= a[j][j]
        for i in range(j + 1, n):
            f = a[i][j] / a[j][j]
            if f:
                for l in range(j, n):
                    a[i][l] -= f * a[j][l]
    return det


def frac_to_dec(x: Fraction) -> Decimal:
    return Decimal(x.numerator) / Decimal(x.denominator)


def I_minus_OZ(O: np.ndarray, mask: int):
    """Exact I - O_Z (xxpp) for the modes in `mask` as Fractions."""
    k = O.shape[0] // 2
    modes = [j for j in range(k) if mask >> j & 1]
    idx = modes + [k + j for j in modes]
    n = len(idx)
    return [[(Fraction(1) if a == b else Fraction(0)) - Fraction(float(O[idx[a], idx[b]]))
             for b in range(n)] for a in range(n)]


def tor_exact(O: np.ndarray) -> Decimal:
    """Eq. 2 with exact determinants and 80-digit square roots."""
    k = O.shape[0] // 2
    total = Decimal(0)
    for mask in range(1 << k):
        m = bin(mask).count("1")
        d = det_exact(I_minus_OZ(O, mask)) if m else Fraction(1)
        t = Decimal(1) / frac_to_dec(d).sqrt()
        total += t if (k - m) % 2 == 0 else -t
    return total


def vacuum_prob_formula(Sigma: np.ndarray, pattern) -> Decimal:
    """Click probability from vacuum probabilities of Sigma (no O involved).

    p(S) = sum over Z subset of S of (-1)^|Z| * P(modes (not S) u Z all in vacuum),
    with P(T all vacuum) = 1/sqrt(det Sigma_T): inclusion-exclusion over the
    clicked modes.  Exact dets of Sigma's own submatrices.
    """
    M = Sigma.shape[0] // 2
    S = [j for j in range(M) if pattern[j]]
    notS = [j for j in range(M) if not pattern[j]]
    total = Decimal(0)
    for zmask in range(1 << len(S)):
        Z = [S[i] for i in range(len(S)) if zmask >> i & 1]
        T = sorted(notS + Z)
        if T:
            idx = T + [M + j for j in T]
            sub = [[Fraction(float(Sigma[a, b])) for b in idx] for a in idx]
            pv = Decimal(1) / frac_to_dec(det_exact(sub)).sqrt()
        else:
            pv = Decimal(1)
        total += pv if len(Z) % 2 == 0 else -pv
    return total
