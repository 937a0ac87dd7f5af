"""Pins for the oracle's observables (O10), Mie series (O11) and the
DDA-versus-Mie accuracy the paper reports (Secs. 3.2, 4)."""
import math

import numpy as np
import pytest

from oracle import dda, errors, lattice, mie, observables, polarizability, system
from paper_0704_0037_gb300 import inputs


# ------------------------------------------------------------------ Mie

def _mie_mpmath(x, m, nterms):
    """Independent evaluation with mpmath spherical Bessel functions (50 digits)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    x = mpmath.mpf(x)
    m = mpmath.mpc(m)
    mx = m * x

    def psi(n, z):
        return z * mpmath.sqrt(mpmath.pi / (2 * z)) * mpmath.besselj(n + 0.5, z)

    def xi(n, z):
        return z * mpmath.sqrt(mpmath.pi / (2 * z)) * (mpmath.besselj(n + 0.5, z)
                                                       + 1j * mpmath.bessely(n + 0.5, z))

    def dpsi(n, z):
        return mpmath.diff(lambda t: psi(n, t), z)

    def dxi(n, z):
        return mpmath.diff(lambda t: xi(n, t), z)

    a, b = [], []
    for n in range(1, nterms + 1):
        p_mx, dp_mx = psi(n, mx), dpsi(n, mx)
        p_x, dp_x = psi(n, x), dpsi(n, x)
        x_x, dx_x = xi(n, x), dxi(n, x)
        a.append(complex((m * p_mx * dp_x - p_x * dp_mx) / (m * p_mx * dx_x - x_x * dp_mx)))
        b.append(complex((p_mx * dp_x - m * p_x * dp_mx) / (p_mx * dx_x - m * x_x * dp_mx)))
    return np.array(a), np.array(b)


@pytest.mark.parametrize("x,m", [(3.0, 1.5), (3.0, 1.33 + 0.1j), (20.0, 2.0)])
def test_mie_coefficients_against_mpmath(x, m):
    a, b = mie.coefficients(x, m)
    k = min(a.size, 12)
    ar, br = _mie_mpmath(x, m, k)
    assert np.allclose(a[:k], ar, rtol=1e-10, atol=1e-13)
    assert np.allclose(b[:k], br, rtol=1e-10, atol=1e-13)


def test_mie_against_scipy_spherical_bessel():
    from scipy.special import spherical_jn, spherical_yn
    x, m = 5.0, 1.4
    a, b = mie.coefficients(x, m)
    n = np.arange(1, a.size + 1)
    mx = m * x
    psi_x = x * spherical_jn(n, x)
    dpsi_x = spherical_jn(n, x) + x * spherical_jn(n, x, derivative=True)
    xi_x = x * (spherical_jn(n, x) + 1j * spherical_yn(n, x))
    dxi_x = dpsi_x + 1j * (spherical_yn(n, x) + x * spherical_yn(n, x, derivative=True))
    psi_m = mx * spherical_jn(n, mx)
    dpsi_m = spherical_jn(n, mx) + mx * spherical_jn(n, mx, derivative=True)
    ar = (m * psi_m * dpsi_x - psi_x * dpsi_m) / (m * psi_m * dxi_x - xi_x * dpsi_m)
    br = (psi_m * dpsi_x - m * psi_x * dpsi_m) / (psi_m * dxi_x - m * xi_x * dpsi_m)
    assert np.allclose(a, ar, rtol=1e-9, atol=1e-14)
    assert np.allclose(b, br, rtol=1e-9, atol=1e-14)


def test_mie_energy_conservation_and_limits():
    for x, m in [(3.0, 1.5), (40.0, 1.05), (20.0, 2.0)]:
        qe, qs, qa, _ = mie.efficiencies(x, m)
        assert abs(qe - qs) < 1e-10 * qe            # real m: no absorption
    # Rayleigh limit
    x, m = 0.01, 1.5
    qe, qs, _, _ = mie.efficiencies(x, m)
    ray = 8.0 / 3.0 * x ** 4 * abs((m * m - 1) / (m * m + 2)) ** 2
    assert abs(qs / ray - 1) < 1e-3
    # m = 1: no scattering
    a, b = mie.coefficients(3.0, 1.0)
    assert np.abs(a).max() < 1e-14 and np.abs(b).max() < 1e-14
    # absorbing sphere: Q_abs > 0
    assert mie.efficiencies(3.0, 1.5 + 0.1j)[2] > 0


def test_mie_angular_integrals():
    """Q_sca = (1/x^2) int (|S1|^2+|S2|^2) sin t dt; Q_ext = (4/x^2) Re S(0);
    g from the same integral weighted by cos t."""
    x, m = 7.0, 1.33 + 0.01j
    qe, qs, _, g = mie.efficiencies(x, m)
    mu, w = np.polynomial.legendre.leggauss(200)
    S1, S2 = mie.amplitudes(x, m, np.rad2deg(np.arccos(mu)))
    s = np.abs(S1) ** 2 + np.abs(S2) ** 2
    assert abs(np.sum(w * s) / x ** 2 / qs - 1) < 1e-10
    assert abs(np.sum(w * s * mu) / x ** 2 / qs / g - 1) < 1e-9
    S1_0, S2_0 = mie.amplitudes(x, m, [0.0])
    assert abs(S1_0[0] - S2_0[0]) < 1e-12 * abs(S1_0[0])
    assert abs(4 / x ** 2 * S1_0[0].real / qe - 1) < 1e-12


# ------------------------------------------------------------------ observables

def test_quadrature_weights():
    dirs, w = observables.sphere_quadrature(16, 32)
    assert abs(w.sum() - 4 * math.pi) < 1e-12
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0)
    e = np.array([1.0, 0.0, 0.0])
    assert abs(np.sum(w * (1 - (dirs @ e) ** 2)) - 8 * math.pi / 3) < 1e-12


def test_qabs_vanishes_for_real_m_any_P():
    rng = np.random.default_rng(0)
    P = rng.standard_normal((3, 40)) + 1j * rng.standard_normal((3, 40))
    for presc in ("rr", "ldr", "cldr"):
        a = polarizability.alpha_diag(1.6, 0.5, presc, (0, 0, 1), (1, 0, 0))
        alpha = np.repeat(a[:, None], 40, axis=1)
        assert abs(observables.q_abs(P, alpha, 0.5, 2.0)) < 1e-14
    a = polarizability.alpha_diag(1.6, 0.5, "cm")
    alpha = np.repeat(a[:, None], 40, axis=1)
    assert observables.q_abs(P, alpha, 0.5, 2.0) < 0        # CM is not energy consistent


def test_optical_theorem_identity_any_P():
    rng = np.random.default_rng(1)
    pos = rng.standard_normal((30, 3)) * 3
    P = rng.standard_normal((3, 30)) + 1j * rng.standard_normal((3, 30))
    kd, xs = 0.4, 2.5
    prop, pol = np.array([0.0, 0.6, 0.8]), np.array([1.0, 0.0, 0.0])
    e = system.incident_field(pos, kd, prop, pol)
    q1 = observables.q_ext(P, e, kd, xs)
    F = observables.farfield(P, pos, kd, prop[None, :])[0]
    q2 = observables.q_ext_forward(F, pol, kd, xs)
    assert abs(q1 - q2) < 1e-12 * abs(q1)


def test_single_dipole_efficiencies():
    kd, xs = 0.3, 0.3 * (3 / (4 * math.pi)) ** (1 / 3)
    alpha = polarizability.alpha_diag(1.5, kd, "ldr")
    P = alpha[:, None] * np.array([[1.0], [0.0], [0.0]])
    pos = np.zeros((1, 3))
    e = system.incident_field(pos, kd, (0, 0, 1), (1, 0, 0))
    qe = observables.q_ext(P, e, kd, xs)
    assert abs(qe - 4 * kd ** 3 * alpha[0].imag / xs ** 2) < 1e-15
    qs = observables.q_sca_quadrature(P, pos, kd, xs, 12, 24)
    assert abs(qs - 8 / 3 * kd ** 6 * abs(alpha[0]) ** 2 / xs ** 2) < 1e-12 * qs
    assert abs(qe - qs) < 1e-12 * qe                     # RR/LDR single dipole conserves energy


@pytest.mark.parametrize("m,presc", [(1.5, "ldr"), (1.5 + 0.2j, "ldr"), (2.0, "rr")])
def test_energy_balance_exact_solution(m, presc):
    """The exact DDA solution (dense LU) satisfies Q_ext = Q_abs + Q_sca."""
    occ = inputs.sphere(6)
    n_occ = int((occ > 0).sum())
    xs = 1.2
    prob = dda.Problem(occ, [m], lattice.kd_volume_corrected(xs, n_occ))
    res = dda.simulate(prob, xs, presc, pols=((1, 0, 0),), method="dense")
    P = res["P"][0]
    qs = observables.q_sca_quadrature(P, prob.pos, prob.kd, xs, 24, 48)
    assert abs(res["qext"][0] - res["qabs"][0] - qs) < 1e-9 * res["qext"][0]


def test_plane_amplitudes_cross_terms_vanish_for_sphere():
    """The xz plane is a symmetry plane of the discretised sphere: S3 = S4 = 0."""
    occ = inputs.sphere(8)
    n_occ = int((occ > 0).sum())
    xs = 2.0
    prob = dda.Problem(occ, [1.5], lattice.kd_volume_corrected(xs, n_occ))
    th = inputs.angles_deg(19)
    res = dda.simulate(prob, xs, "ldr", method="dense", thetas=th)
    S1, S2, S3, S4 = observables.amplitude_plane(res["F"][0], res["F"][1], th)
    scale = np.abs(S1).max()
    assert np.abs(S3).max() < 1e-12 * scale and np.abs(S4).max() < 1e-12 * scale
    # forward direction: S1(0) = S2(0)
    assert abs(S1[0] - S2[0]) < 1e-12 * abs(S1[0])


@pytest.mark.slow
def test_dda_converges_to_mie_config_sphere16():
    """x = 3, m = 1.5, LDR, 16^3 box (about 11 dipoles per wavelength): the DDA
    errors are of the size the paper quotes for this regime (Sec. 4: a few per
    cent for cross sections, max S11 errors < 0.4 for x < 10), and they shrink
    as the lattice is refined."""
    xs, m = 3.0, 1.5
    th = inputs.angles_deg(181)
    s11_mie = mie.s11(xs, m, th)
    qext_mie = mie.efficiencies(xs, m)[0]
    errs = []
    for n in (16, 24):
        occ = inputs.sphere(n)
        prob = dda.Problem(occ, [m], lattice.kd_volume_corrected(xs, int((occ > 0).sum())))
        res = dda.simulate(prob, xs, "ldr", tol=1e-8, thetas=th)
        qext = 0.5 * (res["qext"][0] + res["qext"][1])
        e_q = errors.rel_error(qext, qext_mie)
        e_max, e_rms = errors.s11_errors(res["s11"], s11_mie)
        errs.append((e_q, e_max, e_rms))
        assert abs(res["qabs"][0]) < 1e-10
    assert errs[0][0] < 0.03 and errs[0][1] < 0.4
    assert errs[1][0] < errs[0][0] and errs[1][2] < errs[0][2]


# ---------------------------------------------------------------- full Mueller matrix, <cos theta>
def test_mueller_sphere_form_from_mie():
    """Sphere amplitudes (S3 = S4 = 0): the Mueller matrix by its Stokes
    definition has the textbook block form M11 = M22 = (|S1|^2 + |S2|^2)/2,
    M12 = M21 = (|S2|^2 - |S1|^2)/2, M33 = M44 = Re(S1 S2^*),
    M34 = -M43 = Im(S2 S1^*), all other elements 0."""
    th = inputs.angles_deg(37)
    S1, S2 = mie.amplitudes(3.0, 1.5 + 0.1j, th)
    z = np.zeros_like(S1)
    M = observables.mueller_from_amplitudes(S1, S2, z, z)
    a, b = np.abs(S1) ** 2, np.abs(S2) ** 2
    ref = np.zeros_like(M)
    ref[:, 0, 0] = ref[:, 1, 1] = 0.5 * (a + b)
    ref[:, 0, 1] = ref[:, 1, 0] = 0.5 * (b - a)
    ref[:, 2, 2] = ref[:, 3, 3] = (S1 * np.conj(S2)).real
    ref[:, 2, 3] = (S2 * np.conj(S1)).imag
    ref[:, 3, 2] = -ref[:, 2, 3]
    assert np.abs(M - ref).max() <= 1e-12 * np.abs(ref).max()


def test_mueller_pure_matrix_identities():
    """Any single amplitude matrix gives a non-depolarising Mueller matrix:
    sum_ij M_ij^2 = 4 M11^2, and M11 >= |M_ij|; J = I gives M = I; swapping
    the two field components (S2 = S1 = 0, S3 = S4 = 1) flips Q and V."""
    rng = np.random.default_rng(11)
    S = rng.standard_normal((4, 50)) + 1j * rng.standard_normal((4, 50))
    M = observables.mueller_from_amplitudes(*S)
    assert np.allclose(np.sum(M ** 2, axis=(1, 2)), 4 * M[:, 0, 0] ** 2, rtol=1e-12)
    assert np.all(M[:, :1, :1] >= np.abs(M).max(axis=(1, 2))[:, None, None] - 1e-12)
    one, zero = np.ones(1), np.zeros(1)
    assert np.allclose(observables.mueller_from_amplitudes(one, one, zero, zero)[0], np.eye(4),
                       atol=1e-14)
    swap = observables.mueller_from_amplitudes(zero, zero, one, one)[0]
    assert np.allclose(swap, np.diag([1.0, -1.0, 1.0, -1.0]), atol=1e-14)


def test_asymmetry_quadrature_against_mie_series():
    """<cos theta> from the far field on the sphere quadrature, with the Mie
    amplitudes as the far field (x-polarised incidence:
    |F|^2 = |S2|^2 cos^2 phi + |S1|^2 sin^2 phi), equals the Mie series g."""
    x, m = 4.0, 1.5 + 0.05j
    dirs, w = observables.sphere_quadrature(64, 16)
    th = np.rad2deg(np.arccos(np.clip(dirs[:, 2], -1, 1)))
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    S1, S2 = mie.amplitudes(x, m, th)
    # a field with the right |F|^2: components along theta_hat and phi_hat
    F = np.stack([S2 * np.cos(phi), S1 * np.sin(phi), np.zeros_like(S1)], axis=1)
    g, gvec = observables.asymmetry_from_farfield(F, dirs, w, (0, 0, 1))
    assert abs(g - mie.efficiencies(x, m)[3]) < 1e-10
    assert abs(gvec[0]) < 1e-12 and abs(gvec[1]) < 1e-12
    # a single dipole scatters symmetrically: g = 0
    P = np.array([[1.0 + 0.5j], [0.0], [0.0]])
    Fd = observables.farfield(P, np.zeros((1, 3)), 0.4, dirs)
    assert abs(observables.asymmetry_from_farfield(Fd, dirs, w, (0, 0, 1))[0]) < 1e-14


def test_ypol_from_xpol_by_rotation_symmetry():
    """Sphere lattice (invariant under the 90 degree rotation about z): the
    y-polarised far field equals the rotated x-polarised one (Sec. 3.1's use
    of the spherical symmetry), to round-off with the exact solutions."""
    occ = inputs.sphere(6)
    xs = 1.5
    prob = dda.Problem(occ, [1.5 + 0.1j], lattice.kd_volume_corrected(xs, int((occ > 0).sum())))
    th = inputs.angles_deg(19)
    res = dda.simulate(prob, xs, "ldr", method="dense")
    Px, Py = res["P"]
    d = observables.plane_dirs(th)
    Fy = observables.farfield(Py, prob.pos, prob.kd, d)
    d_rot = np.stack([d[:, 1], -d[:, 0], d[:, 2]], axis=1)      # R^-1 n
    Fy_sym = observables.ypol_farfield_by_symmetry(observables.farfield(Px, prob.pos, prob.kd, d_rot))
    assert np.abs(Fy_sym - Fy).max() < 1e-12 * np.abs(Fy).max()
    Fx = observables.farfield(Px, prob.pos, prob.kd, d)
    M2 = observables.mueller_plane(Fx, Fy, th)
    Ms = observables.mueller_plane(Fx, Fy_sym, th)
    assert np.abs(M2 - Ms).max() < 1e-12 * np.abs(M2).max()


def test_mie_golden_file_matches_the_oracle():
    """tests/golden/mie_spheres.json (read by the benchmark for its errors
    against Mie) is what tests/golden/make_mie_golden.py computes now."""
    import importlib.util
    import json
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_mie_golden",
                                                  os.path.join(here, "make_mie_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(here, "mie_spheres.json")) as f:
        stored = json.load(f)["spheres"]
    fresh = mod.cases()
    assert len(stored) == len(fresh)
    for a, b in zip(stored, fresh):
        assert (a["x"], a["m"]) == (b["x"], b["m"])
        for k in ("qext", "qsca", "g"):
            assert abs(a[k] - b[k]) <= 1e-12 * abs(b[k])
        assert np.allclose(a["s11"], b["s11"], rtol=1e-12, atol=0)
