"""The C-ABI library loads and exports every entry point include/tc.h declares.

Runs without a GPU: it only resolves symbols (no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(tc_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libtc():
    from paper_1602_02740_gb300 import build, tc
    try:
        build.build()
    except RuntimeError as e:  # nvcc missing
        pytest.skip(str(e))
    return ctypes.CDLL(tc.LIB_PATH)


def test_header_declares_boundary():
    names = declared_functions()
    for n in ("tc_create", "tc_destroy", "tc_mul", "tc_sqr", "tc_mul_batch", "tc_serve_submit",
              "tc_serve_poll", "tc_serve_stats", "tc_strerror", "tc_schoolbook",
              "tc_toom_evaluate", "tc_toom_interpolate"):
        assert n in names


def test_every_declared_symbol_is_exported(libtc):
    from paper_1602_02740_gb300 import tc
    for n in declared_functions():
        assert hasattr(libtc, n), f"{n} declared in tc.h but not exported"
        assert n in tc.EXPORTED, f"{n} has no Python binding"


def test_strerror_without_gpu(libtc):
    libtc.tc_strerror.restype = ctypes.c_char_p
    assert libtc.tc_strerror(0) == b"ok"
    assert b"invalid" in libtc.tc_strerror(-1)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1602_02740_gb300 import tc
    monkeypatch.setattr(tc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(tc, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        tc.lib()


def test_host_argument_checks_without_gpu(libtc):
    """Null handles and sizes are rejected on the host (TC_EINVAL) before any CUDA
    call, so these run on a machine without a GPU."""
    vp = ctypes.c_void_p
    h = vp()
    libtc.tc_pipe_create.argtypes = [vp, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int, vp,
                                     ctypes.POINTER(vp)]
    assert libtc.tc_pipe_create(None, 4, 64, 0, None, ctypes.byref(h)) == -1
    libtc.tc_pipe_submit.argtypes = [vp, vp, vp, vp, vp]
    assert libtc.tc_pipe_submit(None, None, None, None, None) == -1
    libtc.tc_pipe_wait.argtypes = [vp]
    assert libtc.tc_pipe_wait(None) == -1
    libtc.tc_pipe_destroy.argtypes = [vp]
    libtc.tc_pipe_destroy(None)
    libtc.tc_batch_destroy.argtypes = [vp]
    libtc.tc_batch_destroy(None)


def test_leaf_karatsuba_threshold_checked_on_the_host(libtc):
    """The base-case variant setting: 0 (off) or a row length the split can
    take (49 limbs and up); anything else is TC_EINVAL."""
    libtc.tc_set_leaf_karatsuba.argtypes = [ctypes.c_int]
    try:
        assert libtc.tc_set_leaf_karatsuba(-1) == -1
        assert libtc.tc_set_leaf_karatsuba(48) == -1
        assert libtc.tc_set_leaf_karatsuba(0) == 0
        assert libtc.tc_set_leaf_karatsuba(49) == 0
    finally:
        assert libtc.tc_set_leaf_karatsuba(384) == 0


def test_batch_tables_rejected_on_the_host(libtc):
    """Negative or huge offsets and lengths in a packed batch are rejected
    (TC_EINVAL) before the context is used or anything is launched."""
    import numpy as np
    vp = ctypes.c_void_p
    libtc.tc_mul_batch.argtypes = [vp, ctypes.c_size_t, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    libtc.tc_batch_prepare.argtypes = [vp, ctypes.c_size_t, vp, vp, vp, vp, vp, vp,
                                       ctypes.POINTER(vp)]
    fake_ctx = ctypes.create_string_buffer(64)     # never dereferenced: rejected first
    fake_buf = ctypes.create_string_buffer(64)
    good = dict(a_off=[0, 8], a_len=[4, 4], b_off=[0, 8], b_len=[4, 4], o_off=[0, 16])
    for key, bad in (("a_off", -1), ("b_off", -5), ("o_off", -8), ("a_len", -1),
                     ("b_len", -2), ("a_len", (1 << 28) + 1), ("a_off", (1 << 40) + 1)):
        arrs = {k: np.array(v, dtype=np.int64) for k, v in good.items()}
        arrs[key][1] = bad
        p = {k: arrs[k].ctypes.data_as(vp) for k in arrs}
        st = libtc.tc_mul_batch(ctypes.addressof(fake_ctx), 2, ctypes.addressof(fake_buf),
                                p["a_off"], p["a_len"], ctypes.addressof(fake_buf), p["b_off"],
                                p["b_len"], ctypes.addressof(fake_buf), p["o_off"], None, None)
        assert st == -1, (key, bad)
        h = vp()
        st = libtc.tc_batch_prepare(ctypes.addressof(fake_ctx), 2, p["a_off"], p["a_len"],
                                    p["b_off"], p["b_len"], p["o_off"], None, ctypes.byref(h))
        assert st == -1 and not h.value, (key, bad)


def test_ntt_roots_of_unity(libtc):
    """The transform's root for length 2^n has order exactly 2^n modulo
    p = 2^64 - 2^32 + 1 (host-only entry point, no GPU)."""
    p = (1 << 64) - (1 << 32) + 1
    libtc.tc_ntt_root.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    for n in range(0, 33):
        r = ctypes.c_uint64()
        assert libtc.tc_ntt_root(n, ctypes.byref(r)) == 0
        w = r.value
        assert 0 < w < p
        assert pow(w, 1 << n, p) == 1
        if n:
            assert pow(w, 1 << (n - 1), p) == p - 1     # primitive: half the order gives -1
    assert libtc.tc_ntt_root(33, ctypes.byref(ctypes.c_uint64())) == -1


def test_ntt_root_makes_small_roots_powers_of_two(libtc):
    """The transform's root w for 2^n points satisfies w^(2^n / 64) = 8 (n >= 6), so
    every root of unity of order <= 64 it uses is a power of 2 modulo p."""
    p = (1 << 64) - (1 << 32) + 1
    libtc.tc_ntt_root.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    for n in range(6, 33):
        r = ctypes.c_uint64()
        assert libtc.tc_ntt_root(n, ctypes.byref(r)) == 0
        assert pow(r.value, 1 << (n - 6), p) == 8
    assert pow(8, 64, p) == 1 and pow(8, 32, p) == p - 1     # 8 has order exactly 64
