"""GB300-native (sm_103a) Born-preconditioned Helmholtz solvers (NPBS hot path).

The compute path is the CUDA library ``libnpbs.so`` (C ABI in
``include/npbs.h``); :mod:`paper_2603_18527_gb300.capi` is a thin ctypes
binding with the same function names.  Build the library with
:func:`paper_2603_18527_gb300.build.build`.
"""
__all__ = ["capi", "build"]
