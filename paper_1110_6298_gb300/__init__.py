"""GB300-native MW spin spherical harmonic transforms (McEwen & Wiaux 2011).

The compute path lives in the CUDA library ``libmw.so`` (C ABI declared in
``include/mw.h``); :mod:`paper_1110_6298_gb300.mw` is the thin ctypes binding
and :mod:`paper_1110_6298_gb300.autograd` wraps it for torch.autograd.  Importing
this package loads nothing; the binding loads the library on first use and
raises if it is missing -- there is no CPU fallback.
"""
__all__ = ["mw", "workloads"]
