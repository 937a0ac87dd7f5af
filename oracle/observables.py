"""O10: scattering quantities from the dipole polarizations.

Sec. 3.1 computes the extinction efficiency, the asymmetry parameter and the
Mueller matrix in one scattering plane.  The formulas are the standard DDA
ones (not printed in the paper), restated with d = 1, kappa = k d, and the
dimensionless polarization P = beta x of Eq. (3) (so alpha is in units of
d^3 and |E0| = 1).  x_size is the size parameter k a_eff of the particle.

  Q_ext = (4 kappa^3 / x^2) sum_i Im(E_inc,i^* . P_i)
  Q_abs = (4 kappa^3 / x^2) sum_i sum_mu [-Im(1/alpha_mu,i) - (2/3) kappa^3] |P_mu,i|^2
  F(n)  = -i kappa^3 (I - n n) sum_j P_j exp(-i kappa n . r_j)
  Q_sca = (1 / (pi x^2)) \\oint |F|^2 dOmega

With the Bohren-Huffman amplitude matrix and incidence along +z, in the xz
plane (n = (sin t, 0, cos t), theta_hat = (cos t, 0, -sin t)):
  x-polarised incidence: S2 = theta_hat . F, S4 = -y_hat . F
  y-polarised incidence: S3 = -theta_hat . F, S1 = y_hat . F
  S11 = (|S1|^2 + |S2|^2 + |S3|^2 + |S4|^2) / 2
The full 4x4 Mueller matrix follows from its definition: Stokes vectors
(I, Q, U, V) = (|E_par|^2 + |E_perp|^2, |E_par|^2 - |E_perp|^2,
2 Re(E_par E_perp^*), -2 Im(E_par E_perp^*)) of the scattered field
(E_par, E_perp)_s = [[S2, S3], [S4, S1]] (E_par, E_perp)_inc for four incident
states whose Stokes vectors span R^4.  The asymmetry parameter is
<cos theta> = \\oint |F|^2 (n . a) dOmega / \\oint |F|^2 dOmega.
"""
import math

import numpy as np


def q_ext(P, e_inc, kd, x_size):
    """Extinction efficiency from the dipole sum."""
    return 4.0 * kd ** 3 / x_size ** 2 * float(np.sum(np.imag(np.conj(e_inc) * P)))


def q_abs(P, alpha, kd, x_size):
    """Absorption efficiency; alpha is (3, N) (diagonal polarizability)."""
    w = -np.imag(1.0 / alpha) - (2.0 / 3.0) * kd ** 3
    return 4.0 * kd ** 3 / x_size ** 2 * float(np.sum(w * np.abs(P) ** 2))


def farfield(P, pos, kd, dirs):
    """Scattering amplitude F(n) for unit directions dirs (K, 3) -> (K, 3)."""
    dirs = np.asarray(dirs, dtype=np.float64)
    out = np.empty((dirs.shape[0], 3), dtype=np.complex128)
    for k, n in enumerate(dirs):
        ph = np.exp(-1j * kd * (pos @ n))
        s = P @ ph                                    # (3,)
        s = s - n * np.dot(n, s)
        out[k] = -1j * kd ** 3 * s
    return out


def q_ext_forward(F_forward, pol, kd, x_size):
    """Optical theorem: C_ext = (4 pi / k^2) Re(e^* . F(a)), i.e.
    Q_ext = 4 Re(e^* . F(a)) / x^2 in these units."""
    e = np.asarray(pol, dtype=np.complex128)
    return 4.0 / x_size ** 2 * float(np.real(np.sum(np.conj(e) * F_forward)))


def plane_dirs(thetas_deg):
    """Directions in the xz scattering plane for angles in degrees."""
    t = np.deg2rad(np.asarray(thetas_deg, dtype=np.float64))
    return np.stack([np.sin(t), np.zeros_like(t), np.cos(t)], axis=1)


def amplitude_plane(F_xpol, F_ypol, thetas_deg):
    """(S1, S2, S3, S4) in the xz plane from the amplitudes of x- and
    y-polarised incidence along +z."""
    t = np.deg2rad(np.asarray(thetas_deg, dtype=np.float64))
    th = np.stack([np.cos(t), np.zeros_like(t), -np.sin(t)], axis=1)
    yh = np.array([0.0, 1.0, 0.0])
    S2 = np.sum(th * F_xpol, axis=1)
    S4 = -(F_xpol @ yh)
    S3 = -np.sum(th * F_ypol, axis=1)
    S1 = F_ypol @ yh
    return S1, S2, S3, S4


def s11_plane(F_xpol, F_ypol, thetas_deg):
    S1, S2, S3, S4 = amplitude_plane(F_xpol, F_ypol, thetas_deg)
    return 0.5 * (np.abs(S1) ** 2 + np.abs(S2) ** 2 + np.abs(S3) ** 2 + np.abs(S4) ** 2)


def sphere_quadrature(n_theta, n_phi):
    """Gauss-Legendre in cos(theta) x uniform phi: (dirs (K,3), weights (K,))
    with sum(weights) = 4 pi."""
    mu, wmu = np.polynomial.legendre.leggauss(n_theta)
    phi = 2.0 * math.pi * np.arange(n_phi) / n_phi
    st = np.sqrt(1.0 - mu * mu)
    dirs = np.stack([
        (st[:, None] * np.cos(phi)[None, :]).ravel(),
        (st[:, None] * np.sin(phi)[None, :]).ravel(),
        np.repeat(mu, n_phi)], axis=1)
    w = np.repeat(wmu, n_phi) * (2.0 * math.pi / n_phi)
    return dirs, w


def q_sca_quadrature(P, pos, kd, x_size, n_theta, n_phi):
    """Q_sca = (1/(pi x^2)) sum_k w_k |F(n_k)|^2 on a product quadrature."""
    dirs, w = sphere_quadrature(n_theta, n_phi)
    F = farfield(P, pos, kd, dirs)
    return float(np.sum(w * np.sum(np.abs(F) ** 2, axis=1))) / (math.pi * x_size ** 2)


def stokes(e_par, e_perp):
    """Stokes vectors (..., 4) of fields with components (E_par, E_perp)."""
    z = e_par * np.conj(e_perp)
    return np.stack([np.abs(e_par) ** 2 + np.abs(e_perp) ** 2,
                     np.abs(e_par) ** 2 - np.abs(e_perp) ** 2,
                     2.0 * z.real, -2.0 * z.imag], axis=-1)


def mueller_from_amplitudes(S1, S2, S3, S4):
    """(n, 4, 4) Mueller matrices by the definition: the scattered Stokes
    vectors of four incident states (parallel, perpendicular, +45 degree and
    circular) against their incident Stokes vectors."""
    S1, S2, S3, S4 = (np.atleast_1d(np.asarray(v, dtype=np.complex128)) for v in (S1, S2, S3, S4))
    r = 1.0 / math.sqrt(2.0)
    states = [(1.0, 0.0), (0.0, 1.0), (r, r), (r, 1j * r)]
    s_in = np.stack([stokes(np.complex128(a), np.complex128(b)) for a, b in states], axis=1)
    s_out = np.stack([stokes(S2 * a + S3 * b, S4 * a + S1 * b) for a, b in states], axis=2)
    return s_out @ np.linalg.inv(s_in)


def mueller_plane(F_xpol, F_ypol, thetas_deg):
    """Mueller matrix in the xz plane, (n, 4, 4)."""
    return mueller_from_amplitudes(*amplitude_plane(F_xpol, F_ypol, thetas_deg))


def asymmetry_from_farfield(F, dirs, weights, prop):
    """<cos theta> and the vector <n> from far fields F (K, 3) at quadrature
    directions dirs (K, 3) with weights (K,): (g, g_vec)."""
    f2 = np.asarray(weights) * np.sum(np.abs(F) ** 2, axis=1)
    gvec = (f2[:, None] * np.asarray(dirs)).sum(axis=0) / f2.sum()
    return float(gvec @ np.asarray(prop, dtype=np.float64)), gvec


def rotate_z90(v):
    """R v for the rotation by +90 degrees about z: (x, y, z) -> (-y, x, z)."""
    v = np.asarray(v)
    return np.stack([-v[..., 1], v[..., 0], v[..., 2]], axis=-1)


def ypol_farfield_by_symmetry(F_xpol_rotdirs):
    """For a lattice invariant under the +90 degree rotation about the
    incidence axis z, the y-polarised amplitude at n equals R F_xpol(R^-1 n).
    Given F_xpol at the directions R^-1 n, return F_ypol at n."""
    return rotate_z90(F_xpol_rotdirs)
