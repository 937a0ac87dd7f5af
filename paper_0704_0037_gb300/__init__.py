"""GB300-native DDA hot path: FFT-accelerated interaction-matrix product and
complex-symmetric Krylov solvers (Yurkin, Maltsev & Hoekstra, arXiv:0704.0037,
Sec. 2, Eqs. (1)-(3)), as hand-written sm_103a CUDA behind a C-ABI library.

Import ``paper_0704_0037_gb300.dda`` for the thin ctypes binding; importing
this package alone loads nothing.
"""
