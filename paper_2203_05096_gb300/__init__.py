"""GB300-native CSR-k sparse matrix-vector multiplication (Lane & Booth, arXiv 2203.05096).

The compute lives in ``libcsrk.so`` (C ABI in ``include/csrk.h``); :mod:`.csrk` is the thin
binding.  Importing this package does not build or load the library; ``csrk.lib()`` does.
"""
from . import csrk

__all__ = ["csrk"]
