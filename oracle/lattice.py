"""O1/O2: the dipole lattice, particle occupancy and the volume correction.

The paper discretises a sphere on a cubic grid with a given number of dipoles
across the diameter (Sec. 3.1, the lambda/(m d) column of Table 1) and applies
a volume correction so that the dipole set has the volume of the sphere
(Sec. 3.1, the paragraph on spherical symmetry and volume correction).  Only
occupied ("real") dipoles carry unknowns (Sec. 2, memory paragraph).

Conventions (oracle test infrastructure; all lengths in units of the dipole
size d):
* a box of nx*ny*nz cells, array shape (nz, ny, nx), x fastest;
* dipole centre of cell (ix, iy, iz): r_mu = (2*i_mu + 1 - n_mu) / 2, i.e. the
  origin is the box centre;
* occupied dipoles are enumerated in lexicographic order with x fastest.
"""
import math

import numpy as np


def sphere_occupancy(n):
    """Cubic box n^3 with a sphere of diameter n (in dipoles) inscribed.

    Cell (i) is occupied iff its centre lies inside the sphere:
    sum_mu (2 i_mu + 1 - n)^2 <= n^2, an exact integer test (no ties occur).
    Returns a bool array of shape (n, n, n), [iz, iy, ix].
    """
    c = (2 * np.arange(n, dtype=np.int64) + 1 - n) ** 2
    s = c[:, None, None] + c[None, :, None] + c[None, None, :]
    return s <= n * n


def ellipsoid_occupancy(nx, ny, nz):
    """Ellipsoid inscribed in an nx x ny x nz box (semi-axes n_mu/2).

    Occupied iff sum_mu ((2 i_mu + 1 - n_mu) / n_mu)^2 <= 1, evaluated exactly
    in integers after multiplying through by (nx ny nz)^2.
    """
    ix = (2 * np.arange(nx, dtype=np.int64) + 1 - nx) ** 2 * (ny * nz) ** 2
    iy = (2 * np.arange(ny, dtype=np.int64) + 1 - ny) ** 2 * (nx * nz) ** 2
    iz = (2 * np.arange(nz, dtype=np.int64) + 1 - nz) ** 2 * (nx * ny) ** 2
    s = iz[:, None, None] + iy[None, :, None] + ix[None, None, :]
    return s <= (nx * ny * nz) ** 2


def cube_occupancy(nx, ny, nz):
    """Every cell of the box occupied."""
    return np.ones((nz, ny, nx), dtype=bool)


def occupied_indices(occ):
    """Integer lattice indices (N, 3) as columns (ix, iy, iz) of occupied cells,
    in lexicographic order with x fastest."""
    iz, iy, ix = np.nonzero(occ)          # C-order scan => x fastest
    return np.stack([ix, iy, iz], axis=1).astype(np.int64)


def positions(occ):
    """Dipole centres (N, 3) in units of d, origin at the box centre (O1)."""
    nz, ny, nx = occ.shape
    ijk = occupied_indices(occ)
    n = np.array([nx, ny, nz], dtype=np.float64)
    return (2.0 * ijk + 1.0 - n) / 2.0


def kd_volume_corrected(x, n_occ):
    """O2 (Sec. 3.1, volume correction): choose d so that N_occ d^3 equals the
    sphere volume (4/3) pi a^3; with x = k a this gives
    kd = x * (4 pi / (3 N_occ))^(1/3)."""
    return x * (4.0 * math.pi / (3.0 * n_occ)) ** (1.0 / 3.0)


def dipoles_per_wavelength(kd, m):
    """lambda / (|m| d) = 2 pi / (|m| kd): the column of Table 1."""
    return 2.0 * math.pi / (abs(m) * kd)
