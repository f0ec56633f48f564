"""GB300-native 2-D complex Gabor filter bank and localized sliding DFT (arXiv 1704.05231).

The compute path is the C-ABI library ``libgaborbank.so`` (hand-written CUDA for sm_103a);
``paper_1704_05231_gb300.bank`` is a thin ctypes binding over it.  Importing this package is
cheap: the library is loaded on first use of ``GaborBank``.
"""
from __future__ import annotations

__all__ = ["Arena", "GaborBank", "GBError", "load_library"]


def __getattr__(name):
    if name in ("Arena", "GaborBank", "GBError", "load_library"):
        from . import bank
        return getattr(bank, name)
    raise AttributeError(name)
