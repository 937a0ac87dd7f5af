"""O3: dipole polarizability prescriptions and the Jacobi factor beta.

Sec. 2 lists four prescriptions: Clausius-Mossotti, radiative-reaction
correction, lattice dispersion relation (LDR) and corrected LDR (CLDR); the
formulas themselves are in the cited works and are restated here as
mathematics (units: d = 1, so alpha is in units of d^3 and kappa = k d):

  alpha_CM = (3 / 4 pi) (eps - 1) / (eps + 2),          eps = m^2
  RR       : 1/alpha = 1/alpha_CM - (2/3) i kappa^3
  LDR      : 1/alpha = 1/alpha_CM + (b1 + b2 m^2 + b3 S m^2) kappa^2 - (2/3) i kappa^3,
             S = sum_mu (a_mu e_mu)^2  (a propagation, e polarisation)
  CLDR     : diagonal; component mu uses b3 m^2 a_mu^2 in place of b3 S m^2
  b1 = -1.8915316, b2 = 0.1648469, b3 = -1.7700004

Eq. (2): beta_i = sqrt(alpha_i) (principal branch), a diagonal 3x3 tensor.
All prescriptions here are diagonal, so alpha and beta are returned as a
length-3 vector (xx, yy, zz) per material.
"""
import math

import numpy as np

LDR_B1 = -1.8915316
LDR_B2 = 0.1648469
LDR_B3 = -1.7700004

PRESCRIPTIONS = ("cm", "rr", "ldr", "cldr")


def alpha_cm(m):
    eps = complex(m) ** 2
    return 3.0 / (4.0 * math.pi) * (eps - 1.0) / (eps + 2.0)


def alpha_diag(m, kd, prescription, prop=(0.0, 0.0, 1.0), pol=(1.0, 0.0, 0.0)):
    """Diagonal polarizability (3,) complex for one material.

    prop: unit propagation vector a; pol: (possibly complex) unit polarisation e.
    Only LDR (through S) and CLDR (through a_mu^2) depend on them.
    """
    m = complex(m)
    a_cm = alpha_cm(m)
    k2 = kd * kd
    k3 = kd * kd * kd
    rad = -(2.0 / 3.0) * 1j * k3
    p = prescription.lower()
    if p == "cm":
        inv = np.full(3, 1.0 / a_cm, dtype=np.complex128)
    elif p == "rr":
        inv = np.full(3, 1.0 / a_cm + rad, dtype=np.complex128)
    elif p == "ldr":
        a = np.asarray(prop, dtype=np.complex128)
        e = np.asarray(pol, dtype=np.complex128)
        S = np.sum((a * e) ** 2)
        corr = (LDR_B1 + LDR_B2 * m * m + LDR_B3 * S * m * m) * k2
        inv = np.full(3, 1.0 / a_cm + corr + rad, dtype=np.complex128)
    elif p == "cldr":
        a = np.asarray(prop, dtype=np.float64)
        corr = (LDR_B1 + LDR_B2 * m * m + LDR_B3 * m * m * a * a) * k2
        inv = 1.0 / a_cm + corr + rad
    else:
        raise ValueError(f"unknown prescription {prescription!r}")
    return 1.0 / inv


def beta_diag(m, kd, prescription, prop=(0.0, 0.0, 1.0), pol=(1.0, 0.0, 0.0)):
    """Eq. (2): beta = sqrt(alpha), principal branch, componentwise."""
    return np.sqrt(alpha_diag(m, kd, prescription, prop, pol))


def per_dipole(values_per_material, mat_index):
    """Spread a (n_mat, 3) table over dipoles: returns (3, N) (SoA layout).
    mat_index holds 0-based material indices of the occupied dipoles."""
    t = np.asarray(values_per_material)
    return t[np.asarray(mat_index)].T.copy()
