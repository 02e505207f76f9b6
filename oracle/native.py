"""Build and load the oracle's C code (test infrastructure only).

``build()`` compiles ``schoolbook.c`` and ``toom.c`` with the host C compiler
into ``oracle/_build/liboracle.so``; ``schoolbook``, ``schoolbook_batch``,
``toom_mul`` and ``toom_mul_batch`` wrap it through ctypes on numpy uint32
limb arrays.  ctypes releases the GIL during the call, so Python threads can
run several products at once.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "schoolbook.c"), os.path.join(_HERE, "toom.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle C code (plain -O2, portable across x86-64 and Arm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cc = os.environ.get("CC", "gcc")
    subprocess.check_call([cc, "-O2", "-std=gnu99", "-shared", "-fPIC", "-pthread"] + _SRCS
                          + ["-o", tmp])
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
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_toom_mul.argtypes = [u32p, u32p, ctypes.c_size_t, ip, ctypes.c_int, u32p,
                                            ctypes.c_int]
            lib.oracle_toom_mul.restype = ctypes.c_int
            lib.oracle_toom_mul_batch.argtypes = [ctypes.c_size_t, u32p, u32p, ctypes.c_size_t,
                                                  ip, ctypes.c_int, u32p, ctypes.c_int]
            lib.oracle_toom_mul_batch.restype = ctypes.c_int
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


TOOM_ERRORS = {1: "a subtraction went below zero", 2: "a division left a remainder",
               3: "a value did not fit its stated length", 4: "out of memory", 5: "bad plan"}


class OracleError(AssertionError):
    pass


def _plan(plan):
    arr = (ctypes.c_int * max(1, len(plan)))(*[int(B) for B in plan])
    return arr, len(plan)


def toom_mul(a: np.ndarray, b: np.ndarray, plan, threads: int = 1) -> np.ndarray:
    """Exact product of two limb arrays of equal length L (2L limbs) by the C
    recursive Toom-Cook (toom.c) with B = plan[l] at level l; the top level's
    2B-1 products on up to ``threads`` threads.  Raises OracleError if an
    invariant of the method fails."""
    lib = _load()
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    if len(a) != len(b):
        raise ValueError("toom_mul takes operands of equal length")
    out = np.zeros(2 * len(a), dtype=np.uint32)
    arr, nlev = _plan(plan)
    st = lib.oracle_toom_mul(_u32(a), _u32(b), len(a), arr, nlev, _u32(out), int(threads))
    if st:
        raise OracleError(f"oracle Toom-Cook: {TOOM_ERRORS.get(st, st)}")
    return out


def toom_mul_batch(A: np.ndarray, B: np.ndarray, plan, threads: int = 1) -> np.ndarray:
    """Row-wise exact products of (count, L) limb arrays by the C recursive
    Toom-Cook, whole products spread over up to ``threads`` threads."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.uint32)
    B = np.ascontiguousarray(B, dtype=np.uint32)
    count, L = A.shape
    OUT = np.zeros((count, 2 * L), dtype=np.uint32)
    arr, nlev = _plan(plan)
    st = lib.oracle_toom_mul_batch(count, _u32(A), _u32(B), L, arr, nlev, _u32(OUT), int(threads))
    if st:
        raise OracleError(f"oracle Toom-Cook: {TOOM_ERRORS.get(st, st)}")
    return OUT
