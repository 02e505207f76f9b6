"""Thin ctypes binding of ``libtc.so`` (include/tc.h), same names as the C ABI.

Only argument marshalling happens here: torch tensors supply device memory
and streams, every arithmetic step runs in the library's CUDA kernels.  Limb
tensors are ``torch.int32`` holding uint32 bit patterns (or ``torch.uint32``).
The library is loaded from this package directory on first use; if it is
missing the call raises ``RuntimeError`` (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")

TC_OK, TC_EINVAL, TC_ENOMEM, TC_EBUSY, TC_ETIMEOUT, TC_EDEVICE, TC_EPENDING = 0, -1, -2, -3, -4, -5, 1
TC_MAX_LEVELS = 8

_lock = threading.Lock()
_lib = None


class TCError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().tc_strerror(status).decode()
        cuda = lib().tc_last_cuda_error()
        super().__init__(f"{where}: {msg} (status {status}, cuda error {cuda})")


TC_BASE_SCHOOLBOOK, TC_BASE_NTT = 0, 1


class tc_opts(ctypes.Structure):
    """A plan: B per Toom level, then the base product.  As a Python list a
    plan is the B values, followed by "ntt" when the base product is the
    number-theoretic transform (e.g. [16, "ntt"], or ["ntt"] alone)."""
    _fields_ = [("levels", ctypes.c_int), ("B", ctypes.c_int * TC_MAX_LEVELS),
                ("base", ctypes.c_int)]

    @classmethod
    def of(cls, Bs: Sequence) -> "tc_opts":
        o = cls()
        Bs = list(Bs)
        o.base = TC_BASE_SCHOOLBOOK
        if Bs and Bs[-1] == "ntt":
            o.base = TC_BASE_NTT
            Bs = Bs[:-1]
        o.levels = len(Bs)
        for i, B in enumerate(Bs):
            o.B[i] = int(B)
        return o

    def plan(self):
        p = [self.B[i] for i in range(self.levels)]
        return p + ["ntt"] if self.base == TC_BASE_NTT else p


_vp, _sz, _u32p, _i64p, _u8p = (ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p)
_optp = ctypes.POINTER(tc_opts)

_SIGS = {
    "tc_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _sz, ctypes.c_char_p]),
    "tc_destroy": (None, [_vp]),
    "tc_check": (ctypes.c_int, [_vp, _vp]),
    "tc_test_bounded_waits": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "tc_set_leaf_karatsuba": (ctypes.c_int, [ctypes.c_int]),
    "tc_plan_for": (ctypes.c_int, [_vp, _sz, _optp]),
    "tc_scratch_bytes": (ctypes.c_int, [_vp, _sz, _sz, _optp, ctypes.POINTER(ctypes.c_size_t)]),
    "tc_mul": (ctypes.c_int, [_vp, _u32p, _sz, _u32p, _sz, _u32p, _optp, _vp]),
    "tc_sqr": (ctypes.c_int, [_vp, _u32p, _sz, _u32p, _optp, _vp]),
    "tc_mul_batch": (ctypes.c_int, [_vp, _sz, _u32p, _i64p, _i64p, _u32p, _i64p, _i64p, _u32p,
                                    _i64p, _optp, _vp]),
    "tc_mul_batch_dev": (ctypes.c_int, [_vp, _sz, _u32p, _i64p, _i64p, _u32p, _i64p, _i64p, _u32p,
                                        _i64p, _sz, _optp, _vp]),
    "tc_batch_prepare": (ctypes.c_int, [_vp, _sz, _i64p, _i64p, _i64p, _i64p, _i64p, _optp,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "tc_batch_run": (ctypes.c_int, [_vp, _vp, _u32p, _u32p, _u32p, _vp]),
    "tc_batch_check": (ctypes.c_int, [_vp, _vp, _vp]),
    "tc_batch_scratch_bytes": (ctypes.c_size_t, [_vp]),
    "tc_batch_destroy": (None, [_vp]),
    "tc_mul_uniform": (ctypes.c_int, [_vp, _sz, _sz, _u32p, _sz, _u32p, _sz, _u32p, _sz, _optp, _vp]),
    "tc_mul_uniform_host": (ctypes.c_int, [_vp, _sz, _sz, _u32p, _u32p, _u32p, _optp, _vp]),
    "tc_pipe_create": (ctypes.c_int, [_vp, _sz, _sz, ctypes.c_int, _optp,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "tc_pipe_submit": (ctypes.c_int, [_vp, _vp, _u32p, _u32p, _u32p]),
    "tc_pipe_wait": (ctypes.c_int, [_vp]),
    "tc_pipe_destroy": (None, [_vp]),
    "tc_schoolbook": (ctypes.c_int, [_sz, _sz, _u32p, _sz, _u32p, _sz, _u32p, _sz, _vp]),
    "tc_ntt_mul": (ctypes.c_int, [_sz, _sz, _u32p, _sz, _u32p, _sz, _u32p, _sz, _vp, _vp]),
    "tc_ntt_work_bytes": (ctypes.c_size_t, [_sz, _sz]),
    "tc_ntt_root": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
    "tc_toom_evaluate": (ctypes.c_int, [_sz, _sz, ctypes.c_int, _u32p, _sz, _u32p, _sz, _u8p, _vp]),
    "tc_toom_interpolate": (ctypes.c_int, [_sz, _sz, ctypes.c_int, _u32p, _sz, _u8p, _u8p, _u32p,
                                           _sz, _vp, _vp]),
    "tc_toom_interpolate_work_bytes": (ctypes.c_size_t, [_sz, _sz, ctypes.c_int]),
    "tc_toom_interpolate_matrix": (ctypes.c_int, [_sz, _sz, ctypes.c_int, _u32p, _sz, _u8p, _u8p,
                                                  _u32p, _sz, _vp]),
    "tc_interp_matrix_table": (ctypes.c_int, [ctypes.c_int, _i64p, _vp, _vp]),
    "tc_toom_interpolate_noalloc": (ctypes.c_int, [_sz, _sz, ctypes.c_int, _u32p, _sz, _u8p, _u8p,
                                                   _u32p, _sz, _vp]),
    "tc_peak_madc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _u32p, _vp,
                                    ctypes.POINTER(ctypes.c_double)]),
    "tc_serve_submit": (ctypes.c_int, [_vp, _u32p, _sz, _u32p, _sz, _u32p,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "tc_serve_poll": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "tc_serve_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "tc_serve_stop": (ctypes.c_int, [_vp]),
    "tc_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "tc_profile_read": (ctypes.c_int, [_vp, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    "tc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "tc_last_cuda_error": (ctypes.c_int, []),
}

EXPORTED = tuple(_SIGS)


def lib():
    """Load libtc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1602_02740_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != TC_OK:
        raise TCError(status, where)


def _ptr(t) -> int:
    """Device (or host) address of a tensor / numpy array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _opts(plan):
    if plan is None:
        return None
    o = plan if isinstance(plan, tc_opts) else tc_opts.of(plan)
    return ctypes.byref(o)


class Context:
    """Owns a tc_ctx (scratch arena, plan table, serving loop)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, table: Optional[str] = None):
        h = ctypes.c_void_p()
        _check(lib().tc_create(ctypes.byref(h), device, budget_bytes,
                               table.encode() if table else None), "tc_create")
        self.handle = h.value
        self.device = device

    def close(self):
        if self.handle:
            lib().tc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tc_create(device: int = 0, budget_bytes: int = 0, table: Optional[str] = None) -> Context:
    return Context(device, budget_bytes, table)


def tc_destroy(ctx: Context):
    ctx.close()


def tc_check(ctx: Context, stream=None):
    """Wait for `stream`; raise TCError(TC_ETIMEOUT) if a bounded device wait of
    a call on this context gave up since the last check."""
    _check(lib().tc_check(ctx.handle, _stream(stream)), "tc_check")


def tc_plan_for(ctx: Context, limbs: int):
    o = tc_opts()
    _check(lib().tc_plan_for(ctx.handle, limbs, ctypes.byref(o)), "tc_plan_for")
    return o.plan()


def tc_scratch_bytes(ctx: Context, count: int, limbs: int, plan=None) -> int:
    v = ctypes.c_size_t()
    _check(lib().tc_scratch_bytes(ctx.handle, count, limbs, _opts(plan), ctypes.byref(v)),
           "tc_scratch_bytes")
    return v.value


def _empty(n, device):
    import torch
    return torch.empty(n, dtype=torch.int32, device=device)


def tc_mul(ctx: Context, a, b, out=None, plan=None, stream=None):
    """out = a * b (1-D int32 device tensors of limbs); returns out (len(a)+len(b) limbs)."""
    na, nb = a.numel(), b.numel()
    if out is None:
        out = _empty(na + nb, a.device)
    assert out.numel() == na + nb
    _check(lib().tc_mul(ctx.handle, _ptr(a), na, _ptr(b), nb, _ptr(out), _opts(plan),
                        _stream(stream)), "tc_mul")
    return out


def tc_sqr(ctx: Context, a, out=None, plan=None, stream=None):
    na = a.numel()
    if out is None:
        out = _empty(2 * na, a.device)
    _check(lib().tc_sqr(ctx.handle, _ptr(a), na, _ptr(out), _opts(plan), _stream(stream)), "tc_sqr")
    return out


def tc_mul_uniform(ctx: Context, A, B, OUT=None, plan=None, stream=None):
    """Row-wise products of 2-D (count, L) int32 device tensors; OUT is (count, 2L)."""
    count, L = A.shape
    if OUT is None:
        import torch
        OUT = torch.empty((count, 2 * L), dtype=torch.int32, device=A.device)
    _check(lib().tc_mul_uniform(ctx.handle, count, L, _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                                _ptr(OUT), OUT.stride(0), _opts(plan), _stream(stream)),
           "tc_mul_uniform")
    return OUT


def tc_mul_uniform_host(ctx: Context, A, B, OUT, plan=None, stream=None):
    """Host-memory variant: A, B (count, L) and OUT (count, 2L) are CPU tensors/arrays."""
    count, L = A.shape
    _check(lib().tc_mul_uniform_host(ctx.handle, count, L, _ptr(A), _ptr(B), _ptr(OUT),
                                     _opts(plan), _stream(stream)), "tc_mul_uniform_host")
    return OUT


class Pipe:
    """Pipelined host-buffer batches (tc_pipe_*): two batches in flight, copies
    overlapping the kernels.  Host buffers handed to submit() must stay alive and
    untouched until wait() returns."""

    def __init__(self, ctx: Context, count: int, limbs: int, square: bool = False, plan=None):
        self.ctx = ctx
        self.count, self.limbs, self.square = count, limbs, square
        h = ctypes.c_void_p()
        _check(lib().tc_pipe_create(ctx.handle, count, limbs, 1 if square else 0, _opts(plan),
                                    ctypes.byref(h)), "tc_pipe_create")
        self.handle = h.value
        self._held = []

    def submit(self, A, B, OUT):
        """A, B (count, limbs) and OUT (count, 2 limbs): contiguous host tensors/arrays."""
        for x, cols in ((A, self.limbs), (OUT, 2 * self.limbs)) + (() if self.square else ((B, self.limbs),)):
            if tuple(x.shape) != (self.count, cols):
                raise ValueError(f"shape {tuple(x.shape)} != {(self.count, cols)}")
            if not (x.flags.c_contiguous if isinstance(x, np.ndarray) else x.is_contiguous()):
                raise ValueError("pipe buffers must be contiguous")
        self._held.append((A, B, OUT))
        _check(lib().tc_pipe_submit(self.ctx.handle, self.handle, _ptr(A),
                                    _ptr(A if self.square else B), _ptr(OUT)), "tc_pipe_submit")
        return OUT

    def wait(self):
        _check(lib().tc_pipe_wait(self.handle), "tc_pipe_wait")
        self._held.clear()

    def close(self):
        if self.handle:
            lib().tc_pipe_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_pipe_create(ctx: Context, count: int, limbs: int, square: bool = False, plan=None) -> Pipe:
    return Pipe(ctx, count, limbs, square, plan)


def tc_mul_batch(ctx: Context, A, a_off, a_len, B, b_off, b_len, OUT, out_off, plan=None,
                 stream=None):
    """Packed batch; offsets/lengths are host int64 numpy arrays."""
    arrs = [np.ascontiguousarray(x, dtype=np.int64) for x in (a_off, a_len, b_off, b_len, out_off)]
    count = len(arrs[0])
    _check(lib().tc_mul_batch(ctx.handle, count, _ptr(A), arrs[0].ctypes.data, arrs[1].ctypes.data,
                              _ptr(B), arrs[2].ctypes.data, arrs[3].ctypes.data, _ptr(OUT),
                              arrs[4].ctypes.data, _opts(plan), _stream(stream)), "tc_mul_batch")
    return OUT


def tc_mul_batch_dev(ctx: Context, A, a_off, a_len, B, b_off, b_len, OUT, out_off, max_limbs: int,
                     plan=None, stream=None):
    """Packed batch with DEVICE int64 offset/length tensors (never read by the host)."""
    for t in (a_off, a_len, b_off, b_len, out_off):
        if not (t.is_cuda and t.dtype.itemsize == 8):
            raise ValueError("tables must be int64 device tensors")
    _check(lib().tc_mul_batch_dev(ctx.handle, a_off.numel(), _ptr(A), _ptr(a_off), _ptr(a_len),
                                  _ptr(B), _ptr(b_off), _ptr(b_len), _ptr(OUT), _ptr(out_off),
                                  int(max_limbs), _opts(plan), _stream(stream)), "tc_mul_batch_dev")
    return OUT


class Batch:
    """A prepared batch (tc_batch_prepare); frees its device tables and scratch on close()."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            lib().tc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_batch_prepare(ctx: Context, a_off, a_len, b_off, b_len, out_off, plan=None) -> Batch:
    """Host-side preparation of a packed batch (offsets/lengths: host int64 arrays)."""
    arrs = [np.ascontiguousarray(x, dtype=np.int64) for x in (a_off, a_len, b_off, b_len, out_off)]
    h = ctypes.c_void_p()
    _check(lib().tc_batch_prepare(ctx.handle, len(arrs[0]), *(x.ctypes.data for x in arrs),
                                  _opts(plan), ctypes.byref(h)), "tc_batch_prepare")
    return Batch(h.value)


def tc_batch_run(ctx: Context, batch: Batch, A, B, OUT, stream=None):
    """Enqueue the prepared batch on `stream` (kernels and memsets only: capturable)."""
    _check(lib().tc_batch_run(ctx.handle, batch.handle, _ptr(A), _ptr(B), _ptr(OUT),
                              _stream(stream)), "tc_batch_run")
    return OUT


def tc_batch_check(ctx: Context, batch: Batch, stream=None):
    _check(lib().tc_batch_check(ctx.handle, batch.handle, _stream(stream)), "tc_batch_check")


def tc_batch_scratch_bytes(batch: Batch) -> int:
    return lib().tc_batch_scratch_bytes(batch.handle)


def tc_batch_destroy(batch: Batch):
    batch.close()


def tc_schoolbook(A, B, OUT=None, stream=None):
    count, L = A.shape
    if OUT is None:
        import torch
        OUT = torch.empty((count, 2 * L), dtype=torch.int32, device=A.device)
    _check(lib().tc_schoolbook(count, L, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(OUT),
                               OUT.stride(0), _stream(stream)), "tc_schoolbook")
    return OUT


def tc_ntt_work_bytes(count: int, limbs: int) -> int:
    return lib().tc_ntt_work_bytes(count, limbs)


def tc_ntt_mul(A, B, OUT=None, work=None, stream=None):
    """Row-wise products of 2-D (count, L) int32 device tensors by the transform
    base product; OUT is (count, 2L).  `work`: device scratch (allocated if None)."""
    import torch
    count, L = A.shape
    if OUT is None:
        OUT = torch.empty((count, 2 * L), dtype=torch.int32, device=A.device)
    if work is None:
        work = torch.empty(max(1, tc_ntt_work_bytes(count, L)), dtype=torch.uint8, device=A.device)
    _check(lib().tc_ntt_mul(count, L, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(OUT),
                            OUT.stride(0), _ptr(work), _stream(stream)), "tc_ntt_mul")
    return OUT


def tc_ntt_root(log2n: int) -> int:
    r = ctypes.c_uint64()
    _check(lib().tc_ntt_root(int(log2n), ctypes.byref(r)), "tc_ntt_root")
    return r.value


def level_sizes(limbs: int, B: int):
    """(b, e, estride, ystride) of one level, as the library lays it out."""
    n = B - 1
    b = -(-limbs // B)
    e = b + -(-(n * (n - 1) + 1) // 32)
    return b, e, -(-e // 4) * 4, -(-2 * e // 4) * 4


def tc_toom_evaluate(U, B: int, OUT=None, SGN=None, stream=None):
    """Evaluate rows of U (count, L) at the 2B-1 points; returns (OUT, SGN)."""
    import torch
    count, L = U.shape
    _, e, estride, _ = level_sizes(L, B)
    if OUT is None:
        OUT = torch.empty((count, 2 * B - 1, estride), dtype=torch.int32, device=U.device)
    if SGN is None:
        SGN = torch.empty((count, 2 * B - 1), dtype=torch.uint8, device=U.device)
    _check(lib().tc_toom_evaluate(count, L, B, _ptr(U), U.stride(0), _ptr(OUT), OUT.shape[-1],
                                  _ptr(SGN), _stream(stream)), "tc_toom_evaluate")
    return OUT, SGN


def tc_toom_interpolate_work_bytes(count: int, limbs: int, B: int) -> int:
    return lib().tc_toom_interpolate_work_bytes(count, limbs, B)


def tc_toom_interpolate(Y, limbs: int, B: int, SGN_U=None, SGN_V=None, OUT=None, work=None,
                        stream=None):
    """Y: (count, 2B-1, ystride) products; returns OUT (count, 2*limbs)."""
    import torch
    count = Y.shape[0]
    if OUT is None:
        OUT = torch.empty((count, 2 * limbs), dtype=torch.int32, device=Y.device)
    wb = tc_toom_interpolate_work_bytes(count, limbs, B)
    if wb and work is None:
        work = torch.empty(wb, dtype=torch.uint8, device=Y.device)
    _check(lib().tc_toom_interpolate(count, limbs, B, _ptr(Y), Y.shape[-1], _ptr(SGN_U), _ptr(SGN_V),
                                     _ptr(OUT), OUT.stride(0), _ptr(work) if wb else None,
                                     _stream(stream)), "tc_toom_interpolate")
    return OUT


def tc_toom_interpolate_matrix(Y, limbs: int, B: int, SGN_U=None, SGN_V=None, OUT=None,
                               stream=None):
    """Interpolation by the inverse Vandermonde matrix (B <= 4, values <= 256 limbs);
    same layout and result as tc_toom_interpolate."""
    import torch
    count = Y.shape[0]
    if OUT is None:
        OUT = torch.empty((count, 2 * limbs), dtype=torch.int32, device=Y.device)
    _check(lib().tc_toom_interpolate_matrix(count, limbs, B, _ptr(Y), Y.shape[-1], _ptr(SGN_U),
                                            _ptr(SGN_V), _ptr(OUT), OUT.stride(0),
                                            _stream(stream)), "tc_toom_interpolate_matrix")
    return OUT


def tc_interp_matrix_table(B: int):
    """Host-side integer form of V^-1 for B blocks: (M[(2B-1), (2B-1)], shift, odd)."""
    npts = 2 * B - 1
    M = np.zeros((npts, npts), dtype=np.int64)
    shift = np.zeros(npts, dtype=np.int32)
    odd = np.zeros(npts, dtype=np.uint32)
    _check(lib().tc_interp_matrix_table(B, M.ctypes.data, shift.ctypes.data, odd.ctypes.data),
           "tc_interp_matrix_table")
    return M, shift, odd


TC_NOALLOC_SCRATCH_BYTES = 16 << 20


def tc_toom_interpolate_noalloc(Y, limbs: int, B: int, SGN_U=None, SGN_V=None, OUT=None,
                                stream=None):
    """tc_toom_interpolate with the library's fixed built-in scratch (no device
    allocation by the library).  For callers that cannot allocate device memory
    while running; the output tensor, if not given, is allocated here by torch
    as a convenience of this binding, not by the library."""
    import torch
    count = Y.shape[0]
    if OUT is None:
        OUT = torch.empty((count, 2 * limbs), dtype=torch.int32, device=Y.device)
    _check(lib().tc_toom_interpolate_noalloc(count, limbs, B, _ptr(Y), Y.shape[-1], _ptr(SGN_U),
                                             _ptr(SGN_V), _ptr(OUT), OUT.stride(0),
                                             _stream(stream)), "tc_toom_interpolate_noalloc")
    return OUT


def tc_serve_submit(ctx: Context, a, b, out) -> int:
    t = ctypes.c_uint64()
    st = lib().tc_serve_submit(ctx.handle, _ptr(a), a.numel(), _ptr(b), b.numel(), _ptr(out),
                               ctypes.byref(t))
    if st == TC_EBUSY:
        return -1
    _check(st, "tc_serve_submit")
    return t.value


def tc_serve_poll(ctx: Context, ticket: int) -> bool:
    st = lib().tc_serve_poll(ctx.handle, ticket)
    if st == TC_EPENDING:
        return False
    _check(st, "tc_serve_poll")
    return True


def tc_serve_stats(ctx: Context):
    p50, p99, bps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_uint64()
    _check(lib().tc_serve_stats(ctx.handle, ctypes.byref(p50), ctypes.byref(p99),
                                ctypes.byref(bps), ctypes.byref(n)), "tc_serve_stats")
    return {"p50_ms": p50.value, "p99_ms": p99.value, "bits_per_s": bps.value,
            "completed": n.value}


def tc_serve_stop(ctx: Context):
    _check(lib().tc_serve_stop(ctx.handle), "tc_serve_stop")


class tc_phase_stat(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("level", ctypes.c_int), ("launches", ctypes.c_int),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("limb_products", ctypes.c_double), ("kernel", ctypes.c_char * 48)]


PHASE_NAMES = {0: "evaluate", 1: "base_case", 2: "interpolate"}


def tc_profile_enable(ctx: Context, on: bool = True):
    _check(lib().tc_profile_enable(ctx.handle, 1 if on else 0), "tc_profile_enable")


def tc_profile_read(ctx: Context):
    """List of dicts: kind, level, kernel, launches, ms, bytes, limb_products."""
    arr = (tc_phase_stat * 64)()
    n = ctypes.c_int()
    _check(lib().tc_profile_read(ctx.handle, arr, 64, ctypes.byref(n)), "tc_profile_read")
    return [{"kind": PHASE_NAMES[a.kind], "level": a.level, "kernel": a.kernel.decode(),
             "launches": a.launches, "ms": a.ms, "bytes": a.bytes,
             "limb_products": a.limb_products} for a in arr[:n.value]]


# ---- limb helpers (numpy uint32 <-> torch int32) ----

def to_device(x: np.ndarray, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).to(device)


def to_numpy(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def tc_peak_madc(blocks: int, iters: int, sink, stream=None) -> float:
    """Enqueue the base case's register-only multiply-accumulate loop; returns
    the number of limb products the launch performs (time it with events)."""
    n = ctypes.c_double()
    _check(lib().tc_peak_madc(int(blocks), int(iters), _ptr(sink), _stream(stream),
                              ctypes.byref(n)), "tc_peak_madc")
    return n.value


def tc_test_bounded_waits(polls: int, withhold: bool):
    """Test hook: shorten the segment-parallel passes' bounded waits to `polls`
    polls (0 = default) and, if `withhold`, make the waits run out."""
    _check(lib().tc_test_bounded_waits(int(polls), 1 if withhold else 0), "tc_test_bounded_waits")


TC_LEAF_KARATSUBA_DEFAULT = 384


def tc_set_leaf_karatsuba(min_limbs: int):
    """Base-case variant: one Karatsuba level inside the lane-pair kernel for
    rows of at least `min_limbs` limbs (0: never; default 384); the same limbs
    either way."""
    _check(lib().tc_set_leaf_karatsuba(int(min_limbs)), "tc_set_leaf_karatsuba")
