"""Large single products: 2^24, 2^26 and 2^27-bit operands, top-level B = 16
and 32 with recursive Toom-Cook below, and squaring at the same sizes.

Every product is compared limb by limb with the oracle's C recursive
Toom-Cook (oracle/toom.c, pinned against CPython and the Python Toom-Cook),
run with the same plan on all host cores; the residues modulo three 61-bit
primes are checked as well.  One 2^24-bit product and one square are also
compared with CPython's integer product."""
import os

import numpy as np
import pytest

from oracle import native, residues
from oracle.limbs import from_int, to_int
from paper_1602_02740_gb300 import inputs

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1

CASES = [
    (1 << 19, [16, 12, 5, 3]), (1 << 19, [32, 8, 5, 3]),
    (1 << 21, [16, 16, 12, 5]), (1 << 21, [32, 16, 8, 4]),
    (1 << 22, [16, 16, 16, 8]), (1 << 22, [32, 16, 12, 5]), (1 << 22, None),
]


def _check(a, b, out, plan):
    assert len(out) == len(a) + len(b)
    want = native.toom_mul(a, b, plan, threads=THREADS)
    if not np.array_equal(out, want):
        bad = np.nonzero(out != want)[0]
        raise AssertionError(f"{len(bad)} limbs differ from the oracle; first at {bad[0]}")
    assert residues.product_residues_match(a, b, out)


@pytest.fixture(scope="module")
def ctx(tc):
    c = tc.tc.tc_create(0)
    yield c
    c.close()


@pytest.mark.parametrize("L,plan", CASES)
def test_large_product(ctx, tc, L, plan):
    t = tc.tc
    a = inputs.uniform(L, L + 3)
    b = inputs.uniform(L, L + 4)
    out = t.to_numpy(t.tc_mul(ctx, t.to_device(a), t.to_device(b), plan=plan))
    _check(a, b, out, plan or t.tc_plan_for(ctx, L))


@pytest.mark.parametrize("L,plan", [(1 << 19, [16, 12, 5, 3]), (1 << 21, [32, 16, 8, 4]),
                                    (1 << 21, [16, 16, 12, 5]), (1 << 22, [16, 16, 16, 8]),
                                    (1 << 22, [32, 16, 12, 5])])
def test_large_square(ctx, tc, L, plan):
    t = tc.tc
    a = inputs.uniform(L, L + 5)
    da = t.to_device(a)
    out = t.to_numpy(t.tc_sqr(ctx, da, plan=plan))
    _check(a, a, out, plan)


def test_large_all_ones_square(ctx, tc):
    # (2^(32L) - 1)^2 = 2^(64L) - 2^(32L+1) + 1, exactly
    t = tc.tc
    L = 1 << 19
    a = inputs.all_ones(L)
    out = t.to_numpy(t.tc_sqr(ctx, t.to_device(a), plan=[16, 12, 5, 3]))
    want = np.zeros(2 * L, dtype=np.uint32)
    want[0] = 1
    want[L] = 0xFFFFFFFE
    want[L + 1:] = 0xFFFFFFFF
    assert np.array_equal(out, want)


@pytest.mark.parametrize("kind", ["equal_halves", "all_ones", "sparse"])
@pytest.mark.parametrize("plan", [[2, 8, 6, 4], [3, 8, 6, 4], [16, 8, 4]])
def test_wide_evaluation_sign_edges(ctx, tc, kind, plan):
    """Top-level evaluation of one long row runs segment-parallel; operands
    whose even and odd parts cancel (U(-1) = 0), or carry everywhere."""
    t = tc.tc
    L = 1 << 16
    if kind == "equal_halves":
        h = inputs.uniform(L // 2, 21)
        a = np.concatenate([h, h])
        b = np.concatenate([h[::-1], h[::-1]]).copy()
    elif kind == "all_ones":
        a = inputs.all_ones(L)
        b = inputs.all_ones(L)
    else:
        a = inputs.sparse(L, 22)
        b = inputs.sparse(L, 23)
    out = t.to_numpy(t.tc_mul(ctx, t.to_device(a), t.to_device(b), plan=plan))
    assert np.array_equal(out, from_int(to_int(a) * to_int(b), 2 * L))


@pytest.mark.parametrize("square", [False, True])
def test_large_product_exact_2e24(ctx, tc, square):
    """Every limb of a 2^24-bit product (the plan table's plan) against CPython."""
    t = tc.tc
    L = 1 << 19
    a = inputs.uniform(L, 91)
    b = a if square else inputs.uniform(L, 92)
    da = t.to_device(a)
    out = t.to_numpy(t.tc_sqr(ctx, da) if square else t.tc_mul(ctx, da, t.to_device(b)))
    want = from_int(to_int(a) * to_int(b), 2 * L)
    assert np.array_equal(out, want)
