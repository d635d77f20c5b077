"""GB300-native BiRank / QuadRank rank queries and QuadFm count-only search.

The CUDA path lives in ``csrc/`` (sm_103a kernels behind the C-ABI declared
in ``include/quadrank.h``); ``capi`` is the thin ctypes binding with the same
entry-point names.  ``synth`` draws the seeded synthetic inputs.
"""
__all__ = ["capi", "synth"]
