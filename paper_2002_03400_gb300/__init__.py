"""GB300-native adaptive randomized butterfly factorization (arXiv:2002.03400).

The compute path is the C-ABI library ``libbutterfly.so`` built from
``csrc/`` (declared in ``include/butterfly.h``); ``api`` is a thin ctypes
binding over it.  ``inputs`` builds seeded synthetic workloads.  Importing
this package does not load the native library; ``api`` does, and raises if
it is missing.
"""
__all__ = ["inputs"]
