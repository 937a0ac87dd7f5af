"""Orientation averaging (Sec. 2, the paragraph on orientation averaging).

The particle orientation is given by Euler angles (alpha, beta, gamma) in the
z-y-z convention: a point r of the particle frame sits at R r in the
laboratory, R = Rz(alpha) Ry(beta) Rz(gamma).  The incident wave travels along
the laboratory z axis, so in the particle frame it propagates along R^T z and
is polarised along R^T x or R^T y; the scattering amplitude transforms as a
vector, F_lab(n) = R F_particle(R^T n).

Averaging over alpha needs no new solution: alpha only turns the scattering
plane about the incidence axis, so the Mueller matrix at azimuth phi of the
scattering plane comes from the two polarisations of the same solution
(parallel = cos phi e_x + sin phi e_y, perpendicular = -sin phi e_x +
cos phi e_y, and amplitudes taken along theta_hat and phi_hat).  Averaging
over beta and gamma needs one pair of solutions per orientation (independent
right-hand sides).  This needs a polarizability that does not depend on the
incident polarisation (CM, RR, CLDR), so that the field of any polarisation is
the same linear combination of the two solutions; LDR's S term depends on it.

The quadrature is fixed (no Romberg adaptivity): Gauss-Legendre in cos(beta),
uniform nodes in gamma and in alpha (the periodic trapezoid rule).
"""
import math

import numpy as np

from . import observables, system


def rot_z(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_y(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def euler_zyz(alpha, beta, gamma):
    return rot_z(alpha) @ rot_y(beta) @ rot_z(gamma)


def grid(n_beta, n_gamma):
    """Orientation nodes (beta, gamma) and weights summing to 1."""
    mu, wmu = np.polynomial.legendre.leggauss(n_beta)
    betas = np.arccos(mu)
    gammas = 2.0 * math.pi * np.arange(n_gamma) / n_gamma
    nodes = [(b, g) for b in betas for g in gammas]
    w = np.array([wb / 2.0 / n_gamma for wb in wmu for _ in gammas])
    return nodes, w


def plane_amplitudes(F_par, F_perp, thetas_deg, phi):
    """(S1, S2, S3, S4) in the plane of azimuth phi (laboratory frame)."""
    t = np.deg2rad(np.asarray(thetas_deg, dtype=np.float64))
    th = np.stack([np.cos(t) * math.cos(phi), np.cos(t) * math.sin(phi), -np.sin(t)], axis=1)
    ph = np.array([-math.sin(phi), math.cos(phi), 0.0])
    S2 = np.sum(th * F_par, axis=1)
    S4 = -(F_par @ ph)
    S3 = -np.sum(th * F_perp, axis=1)
    S1 = F_perp @ ph
    return S1, S2, S3, S4


def oriented(problem, x_size, prescription, R, thetas_deg, n_alpha, solve):
    """Scattering of the particle at orientation R (alpha = 0), with the
    Mueller matrix averaged over n_alpha azimuths of the scattering plane.
    solve(beta, b) -> x.  Returns (Q_ext, Q_abs averaged over the two
    polarisations, M (n, 4, 4))."""
    if prescription.lower() == "ldr":
        raise ValueError("orientation averaging needs a polarisation-independent polarizability")
    a = R.T @ np.array([0.0, 0.0, 1.0])
    eX = R.T @ np.array([1.0, 0.0, 0.0])
    eY = R.T @ np.array([0.0, 1.0, 0.0])
    P, qe, qa = [], [], []
    for e in (eX, eY):
        alpha = problem.alpha(prescription, a, e)
        beta = np.sqrt(alpha)
        b = system.rhs(beta, problem.pos, problem.kd, a, e)
        x = solve(beta, b)
        Pe = beta * x
        P.append(Pe)
        qe.append(observables.q_ext(Pe, system.incident_field(problem.pos, problem.kd, a, e),
                                    problem.kd, x_size))
        qa.append(observables.q_abs(Pe, alpha, problem.kd, x_size))
    t = np.deg2rad(np.asarray(thetas_deg, dtype=np.float64))
    M = np.zeros((t.size, 4, 4))
    for k in range(n_alpha):
        phi = 2.0 * math.pi * k / n_alpha
        n_lab = np.stack([np.sin(t) * math.cos(phi), np.sin(t) * math.sin(phi), np.cos(t)], axis=1)
        n_p = n_lab @ R                                     # rows R^T n
        FX = observables.farfield(P[0], problem.pos, problem.kd, n_p) @ R.T    # R F_p
        FY = observables.farfield(P[1], problem.pos, problem.kd, n_p) @ R.T
        F_par = math.cos(phi) * FX + math.sin(phi) * FY
        F_perp = -math.sin(phi) * FX + math.cos(phi) * FY
        M += observables.mueller_from_amplitudes(*plane_amplitudes(F_par, F_perp, thetas_deg, phi))
    return 0.5 * (qe[0] + qe[1]), 0.5 * (qa[0] + qa[1]), M / n_alpha


def average(problem, x_size, prescription, n_alpha, n_beta, n_gamma, thetas_deg, solve):
    """Orientation-averaged (Q_ext, Q_abs, M (n, 4, 4)) for unpolarised light."""
    nodes, w = grid(n_beta, n_gamma)
    qe = qa = 0.0
    M = 0.0
    for (b, g), wk in zip(nodes, w):
        e, a_, m = oriented(problem, x_size, prescription, euler_zyz(0.0, b, g), thetas_deg,
                            n_alpha, solve)
        qe += wk * e
        qa += wk * a_
        M = M + wk * m
    return qe, qa, M
