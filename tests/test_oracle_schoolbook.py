"""Pins for the oracle's schoolbook product (Section 1: w = u v exactly)."""
import itertools

import numpy as np
import pytest

from oracle import native, residues
from oracle.limbs import from_int, to_int
from paper_1602_02740_gb300 import inputs

EDGE = [0, 1, 1 << 31, 0xFFFFFFFF]


def brute_mul(a: int, b: int) -> int:
    """Shift-and-add over the bits of b: a different algorithm from the oracle's."""
    acc = 0
    i = 0
    while b:
        if b & 1:
            acc += a << i
        b >>= 1
        i += 1
    return acc


def _all_small():
    for L in (1, 2, 3):
        for limbs in itertools.product(EDGE, repeat=L):
            yield np.array(limbs, dtype=np.uint32)


def test_brute_force_tiny_edge_limbs():
    vals = list(_all_small())
    for a in vals:
        for b in vals:
            out = native.schoolbook(a, b)
            assert len(out) == len(a) + len(b)
            assert to_int(out) == brute_mul(to_int(a), to_int(b))


@pytest.mark.parametrize("abits,bbits", [(1, 1), (31, 33), (32, 32), (64, 1), (95, 97),
                                         (1000, 777), (4096, 4095), (12345, 6789)])
def test_closed_form_mersenne(abits, bbits):
    # (2^a - 1)(2^b - 1) = 2^(a+b) - 2^a - 2^b + 1
    La, Lb = -(-abits // 32), -(-bbits // 32)
    a = from_int((1 << abits) - 1, La)
    b = from_int((1 << bbits) - 1, Lb)
    want = (1 << (abits + bbits)) - (1 << abits) - (1 << bbits) + 1
    assert to_int(native.schoolbook(a, b)) == want


@pytest.mark.parametrize("L", [1, 2, 7, 64, 343, 1024])
def test_closed_form_all_ones_square(L):
    # (2^(32L) - 1)^2 = 2^(64L) - 2^(32L+1) + 1
    a = inputs.all_ones(L)
    want = (1 << (64 * L)) - (1 << (32 * L + 1)) + 1
    assert to_int(native.schoolbook(a, a)) == want


@pytest.mark.parametrize("x,y", [(0, 0), (5, 77), (100, 3), (1000, 999)])
def test_closed_form_powers_of_two(x, y):
    a = from_int(1 << x, x // 32 + 1)
    b = from_int(1 << y, y // 32 + 1)
    assert to_int(native.schoolbook(a, b)) == 1 << (x + y)


@pytest.mark.parametrize("L", [1, 5, 300])
def test_zero_and_one(L):
    u = inputs.uniform(L, seed=3)
    zero = np.zeros(L, dtype=np.uint32)
    one = from_int(1, 1)
    assert to_int(native.schoolbook(u, zero)) == 0
    out = native.schoolbook(u, one)
    assert to_int(out) == to_int(u) and len(out) == L + 1


@pytest.mark.parametrize("La,Lb,seed", [(1, 1, 0), (17, 5, 1), (256, 256, 2), (1024, 333, 3),
                                        (4096, 4096, 4)])
def test_residues_and_library_multiply(La, Lb, seed):
    a = inputs.uniform(La, seed)
    b = inputs.uniform(Lb, seed + 100)
    out = native.schoolbook(a, b)
    assert residues.product_residues_match(a, b, out)
    assert to_int(out) == to_int(a) * to_int(b)      # CPython int multiply


def test_residue_check_detects_single_bit_error():
    a = inputs.uniform(200, 9)
    b = inputs.uniform(200, 10)
    out = native.schoolbook(a, b)
    bad = out.copy()
    bad[123] ^= np.uint32(1 << 17)
    assert residues.product_residues_match(a, b, out)
    assert not residues.product_residues_match(a, b, bad)


def test_primes_are_distinct_61_bit_primes():
    ps = residues.primes61()
    assert len(set(ps)) == 3
    for p in ps:
        assert p.bit_length() == 61 and residues.is_prime(p)
    assert (1 << 61) - 1 in ps
    # Miller-Rabin sanity: known composites and primes
    assert not residues.is_prime(561) and not residues.is_prime((1 << 61) - 2)
    assert residues.is_prime(2 ** 31 - 1)


def test_batch_layout_matches_single():
    la = np.array([3, 10, 1, 64], dtype=np.int64)
    lb = np.array([5, 10, 7, 1], dtype=np.int64)
    a_off = np.concatenate([[0], np.cumsum(la)[:-1]])
    b_off = np.concatenate([[0], np.cumsum(lb)[:-1]])
    o_off = np.concatenate([[0], np.cumsum(la + lb)[:-1]])
    A = inputs.uniform(int(la.sum()), 1)
    B = inputs.uniform(int(lb.sum()), 2)
    OUT = native.schoolbook_batch(A, a_off, la, B, b_off, lb, o_off, int((la + lb).sum()))
    for k in range(4):
        a = A[a_off[k]:a_off[k] + la[k]]
        b = B[b_off[k]:b_off[k] + lb[k]]
        assert to_int(OUT[o_off[k]:o_off[k] + la[k] + lb[k]]) == to_int(a) * to_int(b)
