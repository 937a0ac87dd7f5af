"""A whole DDA simulation assembled from the oracle's parts (Sec. 2, Eq. 3).

Lattice (O1/O2) -> polarizability and beta (O3) -> b = beta E_inc (Eq. 3) ->
solve A x = b with the chosen solver (O9) using either the dense matrix, the
brute-force product (O6) or the FFT product (O7) -> P = beta x ->
observables (O10).  Used by the tests and by the CPU baseline leg of the
benchmark; never by the library.
"""
import numpy as np

from . import lattice, observables, polarizability, solvers, system
from .fft_matvec import dmatrix_full, matvec_fft, smooth_size


class Problem:
    """One particle: occupancy (nz, ny, nx) of material indices (0 = void,
    k >= 1 = material k), refractive indices m[k-1], and kd."""

    def __init__(self, occ, m_list, kd, grid=None):
        occ = np.asarray(occ)
        self.occ_mat = occ.astype(np.int64)
        self.occ = occ > 0
        self.nz, self.ny, self.nx = occ.shape
        self.pos = lattice.positions(self.occ)
        self.mat = self.occ_mat[self.occ] - 1          # 0-based, lexicographic order
        self.n_occ = self.pos.shape[0]
        self.m_list = [complex(v) for v in m_list]
        self.kd = float(kd)
        if grid is None:
            grid = tuple(smooth_size(2 * n - 1) for n in (self.nx, self.ny, self.nz))
        self.grid = grid
        self._dmat = None

    def alpha(self, prescription, prop, pol):
        tab = np.stack([polarizability.alpha_diag(m, self.kd, prescription, prop, pol)
                        for m in self.m_list])
        return polarizability.per_dipole(tab, self.mat)

    def beta(self, prescription, prop, pol):
        return np.sqrt(self.alpha(prescription, prop, pol))

    def dmat(self):
        if self._dmat is None:
            self._dmat = dmatrix_full((self.nx, self.ny, self.nz),
                                      (self.grid[0], self.grid[1], self.grid[2]), self.kd)
        return self._dmat

    def matvec(self, beta, method="fft"):
        if method == "fft":
            d = self.dmat()
            return lambda v: matvec_fft(self.occ, beta, d, v)
        if method == "brute":
            return lambda v: system.matvec_bruteforce(self.pos, beta, self.kd, v)
        raise ValueError(method)


def simulate(problem, x_size, prescription="ldr", prop=(0, 0, 1), pols=((1, 0, 0), (0, 1, 0)),
             solver="qmr_cs", tol=1e-5, maxiter=10000, method="fft", thetas=None):
    """Solve Eq. (3) for each polarisation and return the observables.

    Returns dict with per-polarisation P, info, Q_ext, Q_abs, and (when
    thetas is given and both x- and y-polarisations along z are solved)
    S11 in the xz plane."""
    out = dict(P=[], info=[], qext=[], qabs=[], F=[])
    for pol in pols:
        alpha = problem.alpha(prescription, prop, pol)
        beta = np.sqrt(alpha)
        b = system.rhs(beta, problem.pos, problem.kd, prop, pol)
        if method == "dense":
            x = system.solve_dense(problem.pos, beta, problem.kd, b)
            info = dict(status="ok", iters=0, matvecs=0)
        else:
            mv = problem.matvec(beta, method)
            x, info = solvers.SOLVERS[solver](mv, b, tol=tol, maxiter=maxiter)
        P = beta * x
        e_inc = system.incident_field(problem.pos, problem.kd, prop, pol)
        out["P"].append(P)
        out["info"].append(info)
        out["qext"].append(observables.q_ext(P, e_inc, problem.kd, x_size))
        out["qabs"].append(observables.q_abs(P, alpha, problem.kd, x_size))
        if thetas is not None:
            out["F"].append(observables.farfield(P, problem.pos, problem.kd,
                                                 observables.plane_dirs(thetas)))
    if thetas is not None and len(pols) == 2:
        out["s11"] = observables.s11_plane(out["F"][0], out["F"][1], thetas)
    return out
