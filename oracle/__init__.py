"""CPU oracle for the DDA hot path (test infrastructure only).

This package is a plain, slow, obviously-correct complex128 restatement of the
discrete dipole approximation as Yurkin, Maltsev & Hoekstra state it
(arXiv:0704.0037, Sec. 2, Eqs. (1)-(3)), together with the standard
literature formulas the paper cites but does not print (Green's tensor,
polarizability prescriptions, Krylov solvers, far-field observables, Mie
series).  Each function names the passage or formula it follows.

It exists to check the CUDA library, never to stand in for it: only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import it.  It shares no code, table or constant generator
with ``paper_0704_0037_gb300``; neither side imports the other.

Modules
-------
lattice        O1/O2  lattice, sphere/ellipsoid/cube occupancy, volume correction
polarizability O3     CM, RR, LDR, CLDR polarizabilities and beta = sqrt(alpha)
green          O4     free-space Green's tensor
system         O5/O6  dense interaction matrix (Eq. 2), RHS (Eq. 3), brute-force product
fft_matvec     O7/O8  circulant-embedding FFT product with the full (unsymmetrised) D
solvers        O9     QMR-CS, Bi-CG-CS (COCG), Bi-CGSTAB, CGNR
observables    O10    Q_ext, Q_abs, far-field amplitude, S11, Q_sca quadrature
mie            O11    Mie series for a homogeneous sphere
errors         O12    the error measures of Sec. 3.2 (relative Q error, S11 max/RMS)

Parity: every function here is pinned by a ``-m "not gpu"`` test in ``tests/``
against closed forms, invariants, brute force or an independent library
routine; none is marked "parity unpinned" except where stated in its own
docstring.
"""
