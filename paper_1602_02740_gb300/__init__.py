"""Exact B-way Toom-Cook multiplication of large unsigned integers on GB300.

The compute path is the C-ABI library ``libtc.so`` (hand-written sm_103a CUDA
kernels); :mod:`.tc` is its thin ctypes binding.  Importing this package does
not load the library; the first call into :mod:`.tc` does, and raises if it
has not been built.
"""
__all__ = ["tc", "inputs"]


def __getattr__(name):
    if name == "tc":
        from . import tc as _tc
        return _tc
    raise AttributeError(name)
