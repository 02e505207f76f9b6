"""Build and load the oracle's C schoolbook (test infrastructure only).

``build()`` compiles ``schoolbook.c`` with the host C compiler into
``oracle/_build/liboracle.so``; ``schoolbook`` and ``schoolbook_batch`` wrap
it through ctypes on numpy uint32 limb arrays.  ctypes releases the GIL
during the call, so Python threads can run several products at once.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "schoolbook.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle C code (plain -O2, portable across x86-64 and Arm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cc = os.environ.get("CC", "gcc")
    subprocess.check_call([cc, "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_schoolbook.argtypes = [u32p, ctypes.c_size_t, u32p, ctypes.c_size_t, u32p]
            lib.oracle_schoolbook.restype = None
            lib.oracle_schoolbook_batch.argtypes = [
                ctypes.c_size_t, u32p, i64p, i64p, u32p, i64p, i64p, u32p, i64p]
            lib.oracle_schoolbook_batch.restype = None
            _lib = lib
    return _lib


def _u32(x: np.ndarray):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _i64(x: np.ndarray):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def schoolbook(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Exact product of two limb arrays; ``len(a) + len(b)`` limbs."""
    lib = _load()
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    out = np.zeros(len(a) + len(b), dtype=np.uint32)
    if len(a) and len(b):
        lib.oracle_schoolbook(_u32(a), len(a), _u32(b), len(b), _u32(out))
    return out


def schoolbook_batch(A, a_off, a_len, B, b_off, b_len, out_off, out_size) -> np.ndarray:
    """Batched exact products in a packed layout (see schoolbook.c)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.uint32)
    B = np.ascontiguousarray(B, dtype=np.uint32)
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    a_len = np.ascontiguousarray(a_len, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    b_len = np.ascontiguousarray(b_len, dtype=np.int64)
    out_off = np.ascontiguousarray(out_off, dtype=np.int64)
    OUT = np.zeros(out_size, dtype=np.uint32)
    lib.oracle_schoolbook_batch(len(a_off), _u32(A), _i64(a_off), _i64(a_len),
                                _u32(B), _i64(b_off), _i64(b_len), _u32(OUT), _i64(out_off))
    return OUT
