"""Oracle: residue checks of products modulo 61-bit primes.

TEST INFRASTRUCTURE ONLY.

For any size, u v mod p = ((u mod p)(v mod p)) mod p.  Checking a claimed
product against three distinct 61-bit primes costs O(L) and catches any
wrong result except with probability about 2^-180 for a fixed error.  It is a
cheap independent cross-check; bit-exactness is still checked separately.

The primes are 2^61 - 1 (a Mersenne prime) and the two largest primes below
2^61 - 1 that are found by deterministic Miller-Rabin with the first twelve
prime bases (exact for every n < 3.3 * 10^24).
"""
from __future__ import annotations

from functools import lru_cache
from typing import List

from .limbs import to_int

_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24."""
    if n < 2:
        return False
    for p in _BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


@lru_cache(maxsize=None)
def primes61() -> List[int]:
    out = [(1 << 61) - 1]
    c = (1 << 61) - 3
    while len(out) < 3:
        if is_prime(c):
            out.append(c)
        c -= 2
    return out


def residue(limbs, p: int) -> int:
    return to_int(limbs) % p


def product_residues_match(a_limbs, b_limbs, out_limbs) -> bool:
    """True iff out = a * b modulo each of the three primes."""
    A, Bv, W = to_int(a_limbs), to_int(b_limbs), to_int(out_limbs)
    return all((A % p) * (Bv % p) % p == W % p for p in primes61())
