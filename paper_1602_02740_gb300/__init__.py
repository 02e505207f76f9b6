"""Exact B-way Toom-Cook multiplication of large unsigned integers on GB300.

The compute path is the C-ABI library ``libtc.so`` (hand-written sm_103a CUDA
kernels); ``paper_1602_02740_gb300.tc`` is its thin ctypes binding.  Importing
the package does not load the library; the first call into ``tc`` does, and
raises if it has not been built.
"""
