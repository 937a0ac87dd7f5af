"""O7/O8: the circulant-embedding FFT form of the interaction-matrix product.

Sec. 2 (performance paragraph) says the product is done with 3D FFTs (split
into 1D transforms with pruning) and that only the real dipoles carry vector
data.  The mathematics behind it: G depends on r_i - r_j only, so
sum_j G(r_i - r_j) u_j is a linear convolution on the lattice; embedding it in
a periodic grid of M_mu >= 2 n_mu - 1 points per axis (O8) makes it a circular
convolution, computed as IFFT(D ⊙ FFT(pad(u))) with D = FFT(G on the grid).

This oracle keeps the full, unsymmetrised D (6 components x M^3) and plain
scipy.fft 3D transforms: no pruning, no octant storage, no fusion.
"""
import os

import numpy as np
import scipy.fft

from .green import COMPONENTS, green_components

_WORKERS = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def grid_offsets(n, m):
    """Signed lattice offset represented by each grid index 0..m-1 along one
    axis: index j < n -> j, index j > m - n -> j - m, otherwise unused (None
    marked by a mask)."""
    j = np.arange(m)
    off = np.where(j < n, j, j - m).astype(np.float64)
    used = (j < n) | (j > m - n)
    return off, used


def dmatrix_full(shape_n, shape_m, kd):
    """D = FFT3(G sampled at lattice offsets), all 6 components, (6, Mz, My, Mx).

    G at offsets outside |Delta_mu| <= n_mu - 1 is set to zero (those entries
    never multiply valid data when M_mu >= 2 n_mu - 1, O8)."""
    nx, ny, nz = shape_n
    mx, my, mz = shape_m
    if mx < 2 * nx - 1 or my < 2 * ny - 1 or mz < 2 * nz - 1:
        raise ValueError("padded grid must satisfy M >= 2n - 1 on every axis")
    ox, ux = grid_offsets(nx, mx)
    oy, uy = grid_offsets(ny, my)
    oz, uz = grid_offsets(nz, mz)
    dz, dy, dx = np.meshgrid(oz, oy, ox, indexing="ij")
    delta = np.stack([dx, dy, dz], axis=-1)
    mask = uz[:, None, None] & uy[None, :, None] & ux[None, None, :]
    g = green_components(delta, kd)                    # (6, Mz, My, Mx)
    g *= mask[None]
    return scipy.fft.fftn(g, axes=(1, 2, 3), workers=_WORKERS)


def matvec_fft(occ, beta, dmat, x, conj=False):
    """O7: y = x - beta (G (beta x)) via the FFT convolution with the full D.

    occ: (nz, ny, nx) bool occupancy; beta, x: (3, N); dmat from dmatrix_full.
    conj=True returns conj(A conj(x)) = A^H x (A is complex symmetric)."""
    nz, ny, nx = occ.shape
    mz, my, mx = dmat.shape[1:]
    xin = np.conj(x) if conj else x
    u = beta * xin
    grid = np.zeros((3, mz, my, mx), dtype=np.complex128)
    iz, iy, ix = np.nonzero(occ)
    for c in range(3):
        grid[c, iz, iy, ix] = u[c]
    f = scipy.fft.fftn(grid, axes=(1, 2, 3), workers=_WORKERS)
    out = np.zeros_like(f)
    for k, (a, b) in enumerate(COMPONENTS):
        out[a] += dmat[k] * f[b]
        if a != b:
            out[b] += dmat[k] * f[a]
    conv = scipy.fft.ifftn(out, axes=(1, 2, 3), workers=_WORKERS)
    y = xin - beta * conv[:, iz, iy, ix]
    return np.conj(y) if conj else y


def smooth_size(lo, primes=(2, 3, 5, 7)):
    """Smallest integer >= lo whose prime factors all lie in `primes`."""
    m = max(1, int(lo))
    while True:
        r = m
        for p in primes:
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1
