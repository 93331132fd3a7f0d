"""GB300-native hot path of the tracking-enabled island-model genetic
algorithm of arXiv 2404.10861 ("Trackable Agent-based Evolution Models at
Wafer Scale").

The compute lives in ``libhsga.so`` (hand-written CUDA for sm_103a behind a
C-ABI declared in ``include/hsga.h``); :mod:`.binding` marshals arguments to
it with ctypes.  Importing this package loads nothing; the first call into
:mod:`.binding` loads the library and raises if it is missing.
"""
__all__ = ["binding", "inputs"]
