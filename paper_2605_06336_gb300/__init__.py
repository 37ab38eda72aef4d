"""GB300-native angle-dependent parallel-beam CT operators for NL-RMM-GKS.

The compute path is the C-ABI library ``libctgb.so`` (CUDA kernels for
sm_103a); :mod:`paper_2605_06336_gb300.ct` is its thin ctypes binding.
Importing this package loads nothing; the library is opened on first use
and a missing library raises instead of falling back to anything else.
"""
__all__ = ["ct", "synth"]
