"""The transform base product (Toom-Cook over a fast multiply, Section 5) and
Toom-Cook plans over it, limb-exact against the oracle.

tc_ntt_mul multiplies by a number-theoretic transform modulo 2^64 - 2^32 + 1
of the 16-bit digit vectors; its result must equal the plain product bit for
bit at every size: one pass and several passes of the transform, products
whose outputs span several carry segments, all-ones operands (carries through
long runs of 2^32 - 1), squares, and strided rows.
"""
import numpy as np
import pytest

from oracle import native
from oracle.limbs import from_int, to_int
from paper_1602_02740_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(tc):
    c = tc.tc.tc_create(0)
    yield c
    c.close()


SIZES = [1, 2, 3, 7, 16, 33, 64, 100, 255, 256, 257, 1000, 1024, 1025, 2048, 2049, 4096, 5000,
         20000]


@pytest.mark.parametrize("L", SIZES)
@pytest.mark.parametrize("kind", ["uniform", "all_ones", "sparse"])
def test_ntt_mul_vs_oracle(tc, L, kind):
    t = tc.tc
    count = 3 if L <= 5000 else 1
    A = np.stack([inputs.operand(kind, L, 11 * L + k) for k in range(count)])
    B = np.stack([inputs.operand("uniform" if kind == "sparse" else kind, L, 13 * L + k)
                  for k in range(count)])
    out = t.to_numpy(t.tc_ntt_mul(t.to_device(A), t.to_device(B)))
    for k in range(count):
        want = native.schoolbook(A[k], B[k]) if L <= 5000 else from_int(to_int(A[k]) * to_int(B[k]), 2 * L)
        assert np.array_equal(out[k], want), (L, kind, k)


@pytest.mark.parametrize("L", [5, 300, 3000, 9000])
def test_ntt_square_and_strided_rows(tc, L):
    t = tc.tc
    count = 4
    A = np.stack([inputs.uniform(L, 7 * L + k) for k in range(count)])
    A[1] = 0xFFFFFFFF
    dA = t.to_device(np.pad(A, ((0, 0), (0, 4))))[:, :L]      # row stride L + 4
    out = t.to_numpy(t.tc_ntt_mul(dA, dA))                       # squares
    for k in range(count):
        assert np.array_equal(out[k], from_int(to_int(A[k]) ** 2, 2 * L)), (L, k)


def test_ntt_many_products(tc):
    t = tc.tc
    L, count = 700, 3000
    g = inputs.rng(5)
    A = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    B = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    out = t.to_numpy(t.tc_ntt_mul(t.to_device(A), t.to_device(B)))
    for k in list(range(0, count, 97)) + [count - 1]:
        assert np.array_equal(out[k], native.schoolbook(A[k], B[k])), k


# Toom-Cook levels over the transform product (the configuration of Section 5),
# and the transform product alone, through tc_mul.
TOOM_NTT = [(32768, [2, "ntt"]), (32768, [4, "ntt"]), (32768, [12, "ntt"]), (32768, ["ntt"]),
            (1 << 19, [3, "ntt"]), (1 << 19, [16, "ntt"]), (1 << 19, ["ntt"]),
            (1 << 21, [8, "ntt"]), (1 << 22, [4, "ntt"]), (1 << 22, [32, "ntt"]),
            (1 << 22, ["ntt"]), (3000, [3, 2, "ntt"])]


@pytest.mark.parametrize("L,plan", TOOM_NTT)
def test_toom_over_ntt_vs_oracle(ctx, tc, L, plan):
    t = tc.tc
    a = inputs.uniform(L, L + 31)
    b = inputs.uniform(L, L + 32)
    out = t.to_numpy(t.tc_mul(ctx, t.to_device(a), t.to_device(b), plan=plan))
    t.tc_check(ctx)
    # the oracle's own Toom-Cook plan (the product does not depend on the plan)
    oplan = [12, 6, 4] if L <= 32768 else [16, 8, 5, 3] if L <= (1 << 19) else [16, 16, 8, 4]
    want = native.toom_mul(a, b, oplan, threads=8) if L > 5000 else native.schoolbook(a, b)
    assert np.array_equal(out, want), (L, plan)


@pytest.mark.parametrize("L,plan", [(1 << 19, [16, "ntt"]), (1 << 21, ["ntt"])])
def test_toom_over_ntt_square(ctx, tc, L, plan):
    t = tc.tc
    a = inputs.uniform(L, L + 41)
    a[:7] = 0xFFFFFFFF
    da = t.to_device(a)
    out = t.to_numpy(t.tc_sqr(ctx, da, plan=plan))
    want = native.toom_mul(a, a, [16, 8, 4], threads=8)
    assert np.array_equal(out, want)


def test_toom_over_ntt_batch(ctx, tc):
    """A batch at the 2^20-bit benchmark shape with Toom-12 over the transform."""
    t = tc.tc
    L, count = 32768, 24
    A = np.stack([inputs.uniform(L, 300 + 2 * k) for k in range(count)])
    B = np.stack([inputs.uniform(L, 301 + 2 * k) for k in range(count)])
    A[2] = 0xFFFFFFFF
    B[2] = 0xFFFFFFFF
    OUT = t.to_numpy(t.tc_mul_uniform(ctx, t.to_device(A), t.to_device(B), plan=[12, "ntt"]))
    want = native.toom_mul_batch(A, B, [12, 6, 4], threads=8)
    assert np.array_equal(OUT, want)
