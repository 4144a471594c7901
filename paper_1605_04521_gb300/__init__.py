"""GB300-native ORAS-preconditioned FGMRES for high-order Nedelec discretisations of the
time-harmonic Maxwell equations (Bonazzoli, Dolean, Rapetti, Tournier, arXiv:1605.04521).

The product is the C-ABI library built from csrc/ (include/oras.h); `oras` is its ctypes
binding and `build` compiles it in-tree for sm_103a.  Import `paper_1605_04521_gb300.oras`
only after building: it raises if the shared object is missing (there is no fallback).
"""
__all__ = ["build", "oras"]
