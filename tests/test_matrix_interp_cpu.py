"""The integer form of V^-1 that the matrix interpolation uses (host only, no
GPU): every entry equals the oracle's exact Gauss-Jordan inverse (end of
Section 3), the denominators are the smallest that make each row integral,
and applied to true point values it gives the oracle's coefficients."""
from fractions import Fraction
from math import gcd

import pytest

from oracle import toom, vandermonde
from oracle.limbs import to_int
from paper_1602_02740_gb300 import inputs


@pytest.fixture(scope="module")
def tcmod():
    from paper_1602_02740_gb300 import build, tc
    try:
        build.build()
    except RuntimeError as e:  # nvcc missing
        pytest.skip(str(e))
    return tc


@pytest.mark.parametrize("B", [2, 3, 4, 5, 6])
def test_table_equals_oracle_inverse(tcmod, B):
    M, shift, odd = tcmod.tc_interp_matrix_table(B)
    Vi = vandermonde.inverse(tuple(vandermonde.points(B)))
    npts = 2 * B - 1
    for i in range(npts):
        D = (1 << int(shift[i])) * int(odd[i])
        assert int(odd[i]) % 2 == 1
        for p in range(npts):
            assert Fraction(int(M[i, p]), D) == Vi[i][p], (B, i, p)
        # smallest denominator: no common factor left between D and the row
        g = 0
        for p in range(npts):
            g = gcd(g, int(M[i, p]))
        assert gcd(g, D) == 1, (B, i)


def test_table_rejects_bad_arguments(tcmod):
    with pytest.raises(tcmod.TCError):
        tcmod.tc_interp_matrix_table(1)
    with pytest.raises(tcmod.TCError):
        tcmod.tc_interp_matrix_table(7)


@pytest.mark.parametrize("B,L", [(2, 10), (3, 40), (4, 457), (5, 100), (6, 300)])
def test_table_applied_to_point_values(tcmod, B, L):
    """w_i = (sum_p M_ip W(x_p)) / (2^s_i d_i) is exact and equals the oracle's
    coefficients; recomposed it is the product."""
    M, shift, odd = tcmod.tc_interp_matrix_table(B)
    for seed in range(3):
        u = to_int(inputs.uniform(L, 500 + seed))
        v = to_int(inputs.uniform(L, 600 + seed))
        b = toom.ceil_div(L, B)
        ue = toom.evaluate(toom.split(u, B, b))
        ve = toom.evaluate(toom.split(v, B, b))
        y = [p * q for p, q in zip(ue, ve)]
        w = []
        for i in range(2 * B - 1):
            s = sum(int(M[i, p]) * y[p] for p in range(2 * B - 1))
            D = (1 << int(shift[i])) * int(odd[i])
            assert s % D == 0 and s >= 0
            w.append(s // D)
        assert w == vandermonde.interpolate(y, B)
        assert sum(wi << (32 * b * i) for i, wi in enumerate(w)) == u * v
