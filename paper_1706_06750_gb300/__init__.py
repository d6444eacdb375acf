"""KAZE nonlinear scale space and detector on GB300 (sm_103a).

The compute path is the CUDA library ``libkaze.so`` behind the C ABI declared
in ``include/kaze.h``; :mod:`paper_1706_06750_gb300.kaze` is its thin ctypes
binding.  The library is loaded on first use and a missing library is an
error, never a fallback.
"""
__all__ = ["kaze", "synth"]
