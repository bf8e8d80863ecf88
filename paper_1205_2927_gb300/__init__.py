"""GB300-native recursive Strassen-Winograd SGEMM (C = alpha*A*B + beta*C).

The compute path is a C-ABI shared library built from ``csrc/`` for sm_103a;
``paper_1205_2927_gb300.fmm`` is the thin ctypes binding over it.  Importing
this package does not load the library; ``fmm`` does, and fails loudly when
it has not been built.
"""
__all__ = ["inputs"]
