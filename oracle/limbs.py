"""Limb-array <-> Python integer conversion for the oracle (test infrastructure).

A limb array is little-endian ``numpy.uint32``: limb ``i`` holds bits
``[32 i, 32 i + 32)``.  These helpers are the oracle's own; the CUDA path never
converts to Python integers.
"""
from __future__ import annotations

import numpy as np


def to_int(limbs) -> int:
    """Integer value of a little-endian uint32 limb array."""
    a = np.ascontiguousarray(np.asarray(limbs), dtype=np.uint32)
    return int.from_bytes(a.tobytes(), "little")


def from_int(x: int, L: int) -> np.ndarray:
    """``L``-limb little-endian array of ``x`` (0 <= x < 2^(32 L))."""
    if x < 0:
        raise ValueError("negative value has no unsigned limb form")
    if x.bit_length() > 32 * L:
        raise ValueError(f"{x.bit_length()}-bit value does not fit {L} limbs")
    return np.frombuffer(x.to_bytes(4 * L, "little"), dtype=np.uint32).copy()
