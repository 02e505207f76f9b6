"""Oracle: interpolation by exact inversion of the Vandermonde matrix.

TEST INFRASTRUCTURE ONLY.

Section 3 closes with the alternative to the Newton loops: put the powers
x_k^l of the points in a square matrix and invert it.  This module does that
with exact rationals (``fractions.Fraction``) by Gauss-Jordan elimination, for
the 2n+1 points 0, +-1, +-2, ..., +-2^(n-1), and applies the inverse to the
values y_k = W(x_k).  It shares nothing with the Newton/even-odd code, so the
two give independent routes to the coefficients w_0..w_2n.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from typing import List, Sequence, Tuple


def points(B: int) -> List[int]:
    pts = [0]
    for j in range(B - 1):
        pts.append(2 ** j)
        pts.append(-(2 ** j))
    return pts


@lru_cache(maxsize=None)
def inverse(pts: Tuple[int, ...]) -> Tuple[Tuple[Fraction, ...], ...]:
    """Exact inverse of V with V[r][c] = pts[r] ** c (Gauss-Jordan over Q)."""
    N = len(pts)
    M = [[Fraction(p) ** c for c in range(N)] + [Fraction(int(r == i)) for i in range(N)]
         for r, p in enumerate(pts)]
    for col in range(N):
        piv = next(r for r in range(col, N) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        inv_p = 1 / M[col][col]
        M[col] = [x * inv_p for x in M[col]]
        for r in range(N):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    return tuple(tuple(row[N:]) for row in M)


def interpolate(y: Sequence[int], B: int) -> List[int]:
    """Coefficients w_0..w_(2n) of W from W(pts[k]) = y[k]; asserts they are integers."""
    Vi = inverse(tuple(points(B)))
    w = []
    for row in Vi:
        s = sum(c * yk for c, yk in zip(row, y))
        assert s.denominator == 1, "non-integral coefficient"
        w.append(int(s))
    return w
