"""O4: the free-space Green's tensor of Eq. (1).

Eq. (1) uses the complex-symmetric free-space Green's tensor G_ij between
dipoles i and j; its formula is not printed in the paper and is restated from
electrodynamics (units d = 1, kappa = k d, Delta = r_i - r_j, rho = |Delta|):

  G_mu,nu = exp(i kappa rho) / rho^3 *
            [ (kappa^2 rho^2 - 1 + i kappa rho) delta_mu,nu
              - (kappa^2 rho^2 - 3 + 3 i kappa rho) Delta_mu Delta_nu / rho^2 ]

G(0) is defined as 0 (the self term is excluded from the sum in Eq. (1)).
"""
import numpy as np

# component order of the 6 independent entries of the symmetric tensor
COMPONENTS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def green_tensor(delta, kd):
    """G for an array of separations delta (..., 3) -> (..., 3, 3) complex128."""
    d = np.asarray(delta, dtype=np.float64)
    rho2 = np.sum(d * d, axis=-1)
    zero = rho2 == 0.0
    rho2s = np.where(zero, 1.0, rho2)
    rho = np.sqrt(rho2s)
    kr = kd * rho
    pref = np.exp(1j * kr) / (rho2s * rho)
    a = kr * kr - 1.0 + 1j * kr
    b = (kr * kr - 3.0 + 3j * kr) / rho2s
    out = -(b * pref)[..., None, None] * (d[..., :, None] * d[..., None, :])
    idx = np.arange(3)
    out[..., idx, idx] += (a * pref)[..., None]
    out[zero] = 0.0
    return out


def green_components(delta, kd):
    """The 6 independent entries (xx, xy, xz, yy, yz, zz) as (6, ...)."""
    g = green_tensor(delta, kd)
    return np.stack([g[..., m, n] for (m, n) in COMPONENTS], axis=0)


def green_static(delta):
    """kappa -> 0 limit: the static dipole field (3 d^ d^ - I) / rho^3."""
    d = np.asarray(delta, dtype=np.float64)
    rho = np.sqrt(np.sum(d * d, axis=-1))
    u = d / rho[..., None]
    return (3.0 * u[..., :, None] * u[..., None, :] - np.eye(3)) / (rho ** 3)[..., None, None]
