"""Seeded synthetic operands for big-integer multiplication workloads.

This module only draws numbers: it holds none of the multiplication method's
arithmetic.  Both the CUDA path (through the tests and the benchmark) and the
CPU oracle consume what it returns, so it is the one piece of code they share.

Every operand is a little-endian ``numpy.uint32`` limb array: limb ``i`` holds
bits ``[32 i, 32 i + 32)`` of the integer, as in the split of Section 1
(u = U(2^b) with b-bit blocks; here a block is a whole number of limbs).

Workload shapes follow the paper's setting (balanced operands of N bits) and
the synthetic recipes of this library:

* ``uniform``   - limbs uniform over [0, 2^32)
* ``all_ones``  - every limb 0xFFFFFFFF (the maximal-carry operand)
* ``sparse``    - a seeded 1 % of limb positions nonzero, values uniform
* ``batch_lengths`` - log-uniform operand lengths, a fraction unbalanced
* ``poisson_stream`` - arrival times and lengths for a request stream
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "uniform",
    "all_ones",
    "sparse",
    "operand",
    "batch_lengths",
    "poisson_stream",
]


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for ``seed`` (the only source of randomness here)."""
    return np.random.Generator(np.random.PCG64(seed))


def uniform(L: int, seed: int) -> np.ndarray:
    """``L`` limbs drawn uniformly from [0, 2^32)."""
    return rng(seed).integers(0, 1 << 32, size=L, dtype=np.uint64).astype(np.uint32)


def all_ones(L: int) -> np.ndarray:
    """``L`` limbs of 0xFFFFFFFF, i.e. the integer 2^(32 L) - 1."""
    return np.full(L, 0xFFFFFFFF, dtype=np.uint32)


def sparse(L: int, seed: int, frac: float = 0.01) -> np.ndarray:
    """``L`` limbs, ``max(1, round(frac * L))`` seeded positions nonzero."""
    g = rng(seed)
    k = max(1, int(round(frac * L)))
    pos = g.choice(L, size=k, replace=False)
    out = np.zeros(L, dtype=np.uint32)
    out[pos] = g.integers(1, 1 << 32, size=k, dtype=np.uint64).astype(np.uint32)
    return out


def operand(kind: str, L: int, seed: int) -> np.ndarray:
    """Dispatch on ``kind`` in {"uniform", "all_ones", "sparse"}."""
    if kind == "uniform":
        return uniform(L, seed)
    if kind == "all_ones":
        return all_ones(L)
    if kind == "sparse":
        return sparse(L, seed)
    raise ValueError(f"unknown operand kind {kind!r}")


def batch_lengths(count: int, seed: int, lo: int = 64, hi: int = 65536,
                  unbalanced_frac: float = 0.25, max_ratio: float = 4.0):
    """Operand length pairs for a batch of independent products.

    ``La`` is log-uniform in [lo, hi].  A seeded ``unbalanced_frac`` of the
    pairs get ``Lb = ceil(La / r)`` with ``r`` uniform in [1, max_ratio]; a
    coin decides which side is the longer one.  The rest are balanced.
    Returns two int64 arrays (La, Lb).
    """
    g = rng(seed)
    la = np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    la = np.clip(la, lo, hi)
    lb = la.copy()
    unb = g.random(count) < unbalanced_frac
    r = g.uniform(1.0, max_ratio, size=count)
    short = np.maximum(1, np.ceil(la / r)).astype(np.int64)
    swap = g.random(count) < 0.5
    lb = np.where(unb, short, lb)
    a_len = np.where(unb & swap, lb, la)
    b_len = np.where(unb & swap, la, lb)
    return a_len.astype(np.int64), b_len.astype(np.int64)


def poisson_stream(count: int, seed: int, rate_per_s: float, lo: int = 256,
                   hi: int = 1 << 20):
    """Arrival offsets (seconds, cumulative) and balanced operand lengths.

    Inter-arrival gaps are exponential with mean ``1 / rate_per_s``; lengths
    are log-uniform in [lo, hi] limbs.
    """
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    L = np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    return t, np.clip(L, lo, hi)
