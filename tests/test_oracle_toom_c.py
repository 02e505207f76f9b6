"""Pins of the oracle's C recursive Toom-Cook (oracle/toom.c), no GPU.

The C oracle must equal CPython's integer product (a library routine) and the
Python Toom-Cook (oracle/toom.py, independent code on Python integers) on
every plan shape it is used with: B = 2..32, several levels, block sizes that
do not divide the length, all-ones operands (every carry), sparse ones, zero,
and sizes up to 2^22 bits.  Planted mistakes, compiled from edited copies of
toom.c, must be caught by the same comparisons.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import native, toom
from oracle.limbs import from_int, to_int
from paper_1602_02740_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")


def _exact(a, b):
    return from_int(to_int(a) * to_int(b), len(a) + len(b))


PLANS = [
    (1, []), (2, [2]), (3, [3]), (7, [2, 2]), (9, [3]), (16, [4, 2]), (33, [32]),
    (64, [2, 2, 2]), (100, [3, 2]), (129, [5]), (257, [8, 3]), (300, [6, 4]),
    (1000, [12, 3]), (1024, [3]), (1031, [16, 4]), (2048, [32, 2]), (3000, [7, 5]),
    (4096, [12, 6, 4]), (5000, [32, 3]), (6000, [20, 4]), (777, [5, 4, 2]),
]


@pytest.mark.parametrize("L,plan", PLANS)
@pytest.mark.parametrize("kind", ["uniform", "all_ones", "sparse"])
def test_toom_c_equals_cpython(L, plan, kind):
    a = inputs.operand(kind, L, 3 * L + 1)
    b = inputs.operand("uniform" if kind == "sparse" else kind, L, 3 * L + 2)
    assert np.array_equal(native.toom_mul(a, b, plan), _exact(a, b))
    assert np.array_equal(native.toom_mul(a, a, plan), _exact(a, a))   # squares


@pytest.mark.parametrize("L,plan", [(30, [2]), (200, [3, 2]), (500, [8]), (900, [16, 3]),
                                    (1200, [32])])
def test_toom_c_equals_python_toom(L, plan):
    a, b = inputs.uniform(L, L), inputs.uniform(L, L + 7)
    want = toom.toom_multiply(to_int(a), to_int(b), L, plan)
    assert to_int(native.toom_mul(a, b, plan)) == want


def test_toom_c_zero_and_single_top_bit():
    L = 1500
    z = np.zeros(L, np.uint32)
    a = inputs.uniform(L, 5)
    assert not native.toom_mul(z, a, [8, 4]).any()
    t = np.zeros(L, np.uint32)
    t[-1] = 1 << 31
    assert np.array_equal(native.toom_mul(t, t, [16, 3]), _exact(t, t))


def test_toom_c_threads_equal_one_thread():
    L = 20000
    a, b = inputs.uniform(L, 11), inputs.uniform(L, 12)
    one = native.toom_mul(a, b, [12, 6, 4], threads=1)
    assert np.array_equal(native.toom_mul(a, b, [12, 6, 4], threads=5), one)
    A = np.stack([inputs.uniform(600, k) for k in range(9)])
    B = np.stack([inputs.sparse(600, 50 + k) for k in range(9)])
    got = native.toom_mul_batch(A, B, [5, 3], threads=4)
    for k in range(9):
        assert np.array_equal(got[k], _exact(A[k], B[k]))


@pytest.mark.parametrize("L,plan", [(1 << 16, [12, 6, 4]), (1 << 17, [32, 8, 4])])
def test_toom_c_2e21_2e22_bits(L, plan):
    a, b = inputs.uniform(L, 21), inputs.uniform(L, 22)
    assert np.array_equal(native.toom_mul(a, b, plan, threads=os.cpu_count() or 1), _exact(a, b))


def test_toom_c_rejects_bad_plans():
    a = inputs.uniform(10, 1)
    for plan in ([33], [1], [11]):   # B > 32, B < 2, B > L
        with pytest.raises(native.OracleError):
            native.toom_mul(a, a, plan)


# ------------------------------------------------------------------ planted mistakes

MUTANTS = {
    # a wrong index in the evaluation: shift by j(i+1) instead of j i
    "evaluation index": ("(size_t)j * (size_t)i)", "(size_t)j * (size_t)(i + 1))"),
    # a dropped term in Theorem 3.3: k stops one short
    "dropped conversion term": ("for (int k = m; k <= n - 1; ++k) {",
                                "for (int k = m; k < n - 1; ++k) {"),
    # wrong sign in the even-odd combine: W(-x) always taken as positive
    "even-odd sign": ("const int neg = ysgn[2 * k];", "const int neg = 0;"),
    # a transposed operand: the second operand's value at point p taken from point p of u
    "transposed operand": ("if ((st = evaluate(v, L, B, b, e, vval, vs))) goto done;",
                           "if ((st = evaluate(u, L, B, b, e, vval, vs))) goto done;"),
    # wrong node difference in Theorem 3.2: X_(m+k) - X_(m-1)
    "divided-difference node": ("node(pos) - node(m)", "node(pos) - node(m > 0 ? m - 1 : 0)"),
}


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    src = open(os.path.join(ORACLE, "toom.c")).read()
    libs = {}
    d = tmp_path_factory.mktemp("mutants")
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) >= 1, name
        path = d / (re.sub(r"\W+", "_", name) + ".c")
        path.write_text(src.replace(old, new))
        so = d / (path.stem + ".so")
        try:
            subprocess.check_call(["gcc", "-O1", "-std=gnu99", "-shared", "-fPIC", "-pthread",
                                   str(path), os.path.join(ORACLE, "schoolbook.c"), "-o", str(so)])
        except (OSError, subprocess.CalledProcessError) as e:
            pytest.skip(f"no C compiler: {e}")
        lib = ctypes.CDLL(str(so))
        lib.oracle_toom_mul.restype = ctypes.c_int
        libs[name] = lib
    return libs


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(mutant_libs, name):
    lib = mutant_libs[name]
    caught = False
    for L, plan in [(100, [3]), (500, [8, 2]), (1000, [5, 3])]:
        a, b = inputs.uniform(L, L + 1), inputs.uniform(L, L + 2)
        out = np.zeros(2 * L, np.uint32)
        p = (ctypes.c_int * len(plan))(*plan)
        u32 = ctypes.POINTER(ctypes.c_uint32)
        st = lib.oracle_toom_mul(a.ctypes.data_as(u32), b.ctypes.data_as(u32), ctypes.c_size_t(L),
                                 p, len(plan), out.ctypes.data_as(u32), 1)
        if st != 0 or not np.array_equal(out, _exact(a, b)):
            caught = True
    assert caught, f"planted mistake '{name}' not detected"
