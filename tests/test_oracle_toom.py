"""Pins for the oracle's recursive Toom-Cook, step by step.

Every intermediate is checked against something other than the oracle's own
code: the polynomial definitions of Section 1, the explicit Newton formula
(Theorem 3.1, eq. 3.2), exact Vandermonde inversion (end of Section 3), the
block convolution w_k = sum_i u_i v_(k-i), the C schoolbook and CPython's
integer product.  The last tests plant mistakes in copies of oracle steps and
check that these pins catch them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import native, toom, vandermonde
from oracle.limbs import from_int, to_int
from paper_1602_02740_gb300 import inputs


def poly_at(blocks, x):
    return sum(c * x ** i for i, c in enumerate(blocks))


def block_convolution(ub, vb):
    B = len(ub)
    return [sum(ub[i] * vb[k - i] for i in range(B) if 0 <= k - i < B) for k in range(2 * B - 1)]


def newton_alpha_explicit(X, y):
    """eq. 3.2: alpha_k = sum_i y_i / prod_(j != i, j <= k) (X_i - X_j)."""
    out = []
    for k in range(len(X)):
        s = Fraction(0)
        for i in range(k + 1):
            den = 1
            for j in range(k + 1):
                if j != i:
                    den *= X[i] - X[j]
            s += Fraction(y[i], den)
        assert s.denominator == 1
        out.append(int(s))
    return out


def check_level(lt):
    B = lt.B
    pts = toom.eval_points(B)
    assert len(pts) == 2 * B - 1
    for p, x in enumerate(pts):
        assert lt.u_eval[p] == poly_at(lt.u_blocks, x)
        assert lt.v_eval[p] == poly_at(lt.v_blocks, x)
        assert lt.y[p] == lt.u_eval[p] * lt.v_eval[p]
    w_conv = block_convolution(lt.u_blocks, lt.v_blocks)
    assert lt.w == w_conv
    assert vandermonde.interpolate(lt.y, B) == w_conv
    X = toom.nodes(B)
    assert lt.alpha_e == newton_alpha_explicit(X, lt.ye)
    assert lt.alpha_o == newton_alpha_explicit(X, lt.yo)
    # even polynomial W_e(X) = sum w_2i X^i, odd one X W_o(X) = sum w_(2i+1) X^(i+1)
    assert lt.ce == w_conv[0::2]
    assert lt.co == [0] + w_conv[1::2]
    assert lt.result == poly_at(lt.u_blocks, 1 << (32 * lt.b)) * poly_at(lt.v_blocks, 1 << (32 * lt.b))


CASES = [
    # (L, plan)
    (1, [2]), (2, [2]), (5, [3]), (7, [4]), (9, [5]), (40, [8]), (64, [16]), (100, [32]),
    (1024, [3]), (300, [16, 2]), (500, [3, 3, 2]), (777, [32, 3]), (129, [4, 4, 4]),
]


@pytest.mark.parametrize("L,plan", CASES)
@pytest.mark.parametrize("kind", ["uniform", "all_ones", "sparse"])
def test_toom_levels_pinned(L, plan, kind):
    a = inputs.operand(kind, L, seed=L)
    b = inputs.operand(kind, L, seed=L + 7)
    u, v = to_int(a), to_int(b)
    tr = toom.Trace()
    r = toom.toom_multiply(u, v, L, plan, tr)
    assert r == u * v
    assert to_int(native.schoolbook(a, b)) == r
    assert len(tr.levels) == sum(math.prod(2 * B - 1 for B in plan[:l]) for l in range(len(plan)))
    for lt in tr.levels.values():
        check_level(lt)
    for (uu, vv, yy) in tr.leaves.values():
        assert yy == uu * vv


@pytest.mark.parametrize("B", [2, 3, 4, 5, 6, 7, 8, 12, 16, 24, 32])
def test_all_ones_extremes_every_B(B):
    """Maximal blocks drive every intermediate to its largest size; the bound
    assertions inside the oracle (e limbs for evaluations, 2e+1 limbs for the
    interpolation) must hold."""
    L = 3 * B + 1
    a = inputs.all_ones(L)
    u = to_int(a)
    tr = toom.Trace()
    assert toom.toom_multiply(u, u, L, [B], tr) == u * u
    check_level(tr.levels[(0, 0)])


def test_points_and_nodes_section6():
    # Section 6: points 0, 1, 2, 4, ..., 2^(n-1) (and their negatives), so for
    # B = 16 the largest X = x^2 is 2^28 and every divisor fits one 32-bit word.
    B = 16
    pts = toom.eval_points(B)
    assert sorted(p for p in pts if p >= 0) == [0] + [2 ** j for j in range(15)]
    X = toom.nodes(B)
    assert max(X) == 2 ** 28
    for k in range(1, B):
        for m in range(k, B):
            d = X[m] - X[m - k]
            assert 0 < d < 2 ** 32
            odd = d >> ((d & -d).bit_length() - 1)
            assert odd == 4 ** k - 1 or m == k


@pytest.mark.parametrize("L,plan", [(3000, [16]), (5000, [32, 2]), (2048, [8, 4])])
def test_toom_larger_vs_library(L, plan):
    a = inputs.uniform(L, 11)
    b = inputs.uniform(L, 12)
    u, v = to_int(a), to_int(b)
    assert toom.toom_multiply(u, v, L, plan) == u * v


def test_level_sizes_rule():
    # b = ceil(L/B); evaluation length e = b + ceil((n(n-1)+1)/32)
    assert toom.level_sizes(1024, [3]) == [(3, 1024, 342, 343)]
    assert toom.level_sizes(32768, [16, 8]) == [(16, 32768, 2048, 2055), (8, 2055, 257, 259)]
    assert toom.growth_limbs(2) == 1 and toom.growth_limbs(32) == 30


# --------------------------------------------------------------------------
# Planted mistakes: each mutant is a copy of one oracle step with one error;
# the pins above must reject it.
# --------------------------------------------------------------------------

def _interp(y, B, eo=toom.even_odd_combine, dd=toom.divided_differences,
            n2m=toom.newton_to_monomial):
    X = toom.nodes(B)
    ye, yo = eo(y)
    return toom.interleave(n2m(X, dd(X, ye)), n2m(X, dd(X, yo)))


def _eo_wrong_sign(y):
    n = (len(y) - 1) // 2
    ye, yo = [y[0]], [0]
    for k in range(1, n + 1):
        x = 1 << (k - 1)
        ye.append((y[2 * k - 1] - y[2 * k]) // 2)     # sign flipped
        yo.append(x * ((y[2 * k - 1] + y[2 * k]) // 2))
    return ye, yo


def _dd_wrong_index(X, y):
    n = len(X) - 1
    col = list(y)
    for k in range(1, n + 1):
        prev = col
        col = list(prev)
        for pos in range(k, n + 1):
            col[pos] = (prev[pos] - prev[pos - 1]) // (X[pos] - X[pos - 1])   # X_m -> X_(pos-1)
    return col


def _n2m_transposed(X, alpha):
    n = len(X) - 1
    beta = list(alpha)
    for m in range(n - 1, -1, -1):
        old = beta
        beta = list(old)
        for k in range(m, n):
            beta[k] = old[k + 1] - X[m] * old[k]        # operands transposed
    return beta


def _n2m_dropped_term(X, alpha):
    n = len(X) - 1
    beta = list(alpha)
    for m in range(n - 1, 0, -1):                       # m = 0 step dropped (harmless: X_0 = 0)
        old = beta
        beta = list(old)
        for k in range(m, n - 1):                       # last k dropped
            beta[k] = old[k] - X[m] * old[k + 1]
    return beta


def _eval_dropped_term(blocks):
    B = len(blocks)
    vals = [blocks[0]]
    for j in range(B - 1):
        x = 1 << j
        E = sum(c * x ** i for i, c in enumerate(blocks[:-1]) if i % 2 == 0)   # top block lost
        O = sum(c * x ** i for i, c in enumerate(blocks[:-1]) if i % 2 == 1)
        vals += [E + O, E - O]
    return vals


@pytest.mark.parametrize("B", [3, 4, 8])
def test_planted_mistakes_are_caught(B):
    L = 10 * B
    a = inputs.uniform(L, 5)
    b = inputs.uniform(L, 6)
    bsz = toom.ceil_div(L, B)
    ub, vb = toom.split(to_int(a), B, bsz), toom.split(to_int(b), B, bsz)
    y = [p * q for p, q in zip(toom.evaluate(ub), toom.evaluate(vb))]
    w = block_convolution(ub, vb)
    assert _interp(y, B) == w

    def rejected(fn):
        try:
            return fn() != w
        except (AssertionError, ZeroDivisionError):
            return True

    assert rejected(lambda: _interp(y, B, eo=_eo_wrong_sign))
    assert rejected(lambda: _interp(y, B, dd=_dd_wrong_index))
    assert rejected(lambda: _interp(y, B, n2m=_n2m_transposed))
    assert rejected(lambda: _interp(y, B, n2m=_n2m_dropped_term))
    bad_eval = _eval_dropped_term(ub)
    assert any(bad_eval[p] != poly_at(ub, x) for p, x in enumerate(toom.eval_points(B)))


def test_interpolation_intermediates_nonnegative_unit_vectors():
    """Reading of Section 4: with W(x) >= |W(-x)| the even-odd values are >= 0.
    Algorithms 1 and 2 are linear; on the nodes 0,1,4,.. every unit coefficient
    vector gives non-negative intermediates, so every W with non-negative
    coefficients does too."""
    for B in (2, 3, 4, 8, 16, 32):
        n = B - 1
        X = toom.nodes(B)
        for j in range(n + 1):
            coeffs = [int(i == j) for i in range(n + 1)]
            y = [poly_at(coeffs, x) for x in X]
            for state in toom.interpolation_intermediates_all(X, y):
                assert min(state) >= 0
            assert toom.interpolation_intermediates_all(X, y)[-1] == coeffs
