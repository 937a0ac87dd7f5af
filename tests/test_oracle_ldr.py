"""The LDR coefficients b1, b2, b3 of the oracle, derived independently.

Sec. 2 lists the lattice dispersion relation (LDR) polarizability among
ADDA's prescriptions and cites it without printing it.  Its defining
property: an infinite simple cubic lattice of point dipoles (spacing d = 1)
with that polarizability carries a transverse plane wave with the continuum
dispersion relation |k| = m kd, to order (kd)^2.  A Bloch mode P_j =
e exp(i k.r_j) satisfies P = alpha E_loc, so the polarizability that carries
it is

    1/alpha = e . T(kd, k) . e,    T = sum_{r != 0} G(r) exp(i k.r),

with G the free-space dyadic Green's tensor of wavenumber kd.  The LDR writes
1/alpha = 1/alpha_CM + (b1 + b2 m^2 + b3 S m^2) kd^2 - (2/3) i kd^3 with
S = sum_mu (a_mu e_mu)^2 (a = k/|k|).  This test evaluates T by Ewald
summation -- G = (kd^2 + grad grad) exp(i kd R)/R split with erfc into a
real-space sum and a reciprocal-lattice sum -- for several (m, a, e), fits the
coefficient of kd^2 in T - 1/alpha_CM + (2/3) i kd^3 as kd -> 0, and solves
for b1, b2, b3.  A typo in a digit or a sign of the oracle's constants, or a
wrong S term, fails it.  Nothing here is shared with the oracle but its
constants and alpha_diag under test.
"""
import itertools
import json
import os

import numpy as np
import scipy.special as sp

from oracle import polarizability

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ldr_coefficients.json")
SQPI = np.sqrt(np.pi)


def lattice_sum(kd, kvec, e, eta=SQPI, n_real=6, n_recip=6):
    """e . sum_{r in Z^3, r != 0} G(r) exp(i k.r) . e  (unit cubic lattice).

    Ewald split of exp(i kd R)/R = f(R) + L(R) with
      f(R) = [exp(i kd R) erfc(eta R + i kd/(2 eta)) + exp(-i kd R) erfc(eta R - i kd/(2 eta))] / (2R)
    (short range) and L whose Bloch sum is
      4 pi sum_g exp(i (k+g).x) exp(-(|k+g|^2 - kd^2)/(4 eta^2)) / (|k+g|^2 - kd^2).
    G = (kd^2 + grad grad) applied to each part; the r = 0 term of the
    smooth part, -L, is even and analytic in R and contributes kd^2 h0 + 2 h2
    (h = -L = h0 + h2 R^2 + ...)."""
    kvec = np.asarray(kvec, dtype=np.float64)
    e = np.asarray(e, dtype=np.complex128)
    ee = e @ e
    # reciprocal-lattice part at x = 0: 4 pi sum (kd^2 ee - (e.q)^2) E_q / (q^2 - kd^2)
    r1 = np.arange(-n_recip, n_recip + 1)
    q = kvec + 2.0 * np.pi * np.array(list(itertools.product(r1, r1, r1)), dtype=np.float64)
    q2 = np.einsum("ij,ij->i", q, q)
    qe = q @ e
    recip = 4.0 * np.pi * np.sum((kd ** 2 * ee - qe * qe) * np.exp(-(q2 - kd ** 2) / (4 * eta ** 2))
                                 / (q2 - kd ** 2))
    # real-space part: e.(kd^2 + grad grad) f(|x - r|).e at x = 0, r != 0; for a
    # radial f, grad grad f = f'' RR + (f'/R)(I - RR)
    r2 = np.arange(-n_real, n_real + 1)
    r = np.array([v for v in itertools.product(r2, r2, r2) if any(v)], dtype=np.float64)
    R = np.sqrt(np.einsum("ij,ij->i", r, r))
    c = 1j * kd / (2 * eta)
    Ap = np.exp(1j * kd * R) * sp.erfc(eta * R + c)
    Am = np.exp(-1j * kd * R) * sp.erfc(eta * R - c)
    S, D = Ap + Am, Ap - Am
    Q = np.exp(-eta ** 2 * R ** 2 + kd ** 2 / (4 * eta ** 2))  # exp(+-i kd R) exp(-(eta R +- c)^2)
    S1 = 1j * kd * D - (4 * eta / SQPI) * Q
    S2 = -kd ** 2 * S + (8 * eta ** 3 * R / SQPI) * Q
    f = S / (2 * R)
    f1 = S1 / (2 * R) - S / (2 * R ** 2)
    f2 = S2 / (2 * R) - S1 / R ** 2 + S / R ** 3
    er2 = ((r @ e) / R) ** 2
    real = np.sum(np.exp(1j * (r @ kvec)) * (kd ** 2 * f * ee + f2 * er2 + (f1 / R) * (ee - er2)))
    # r = 0: h(R) = (u(R) - u(-R)) / (2R), u = exp(-i kd R) erfc(eta R + c0),
    # h0 = u'(0), h2 = u'''(0) / 6
    c0 = -1j * kd / (2 * eta)
    E0 = np.exp(-c0 * c0)
    w0 = sp.erfc(c0)
    w1 = -(2 * eta / SQPI) * E0
    w2 = (4 * eta ** 2 * c0 / SQPI) * E0
    w3 = -(2 * eta / SQPI) * (-2 * eta ** 2 + 4 * eta ** 2 * c0 * c0) * E0
    ik = -1j * kd
    h0 = ik * w0 + w1
    h2 = (ik ** 3 * w0 + 3 * ik ** 2 * w1 + 3 * ik * w2 + w3) / 6.0
    return recip + real + (kd ** 2 * h0 + 2 * h2) * ee


def inv_alpha_cm(m):
    eps = complex(m) ** 2
    return (4.0 * np.pi / 3.0) * (eps + 2.0) / (eps - 1.0)


def kd2_coefficient(m, a, e, kds=(0.01, 0.015, 0.02, 0.03, 0.04)):
    """Limit kd -> 0 of [T - 1/alpha_CM + (2/3) i kd^3] / kd^2 (fit in kd^2)."""
    a = np.asarray(a, dtype=np.float64)
    a = a / np.linalg.norm(a)
    e = np.asarray(e, dtype=np.complex128)
    e = e / np.linalg.norm(e)
    y = []
    for kd in kds:
        t = lattice_sum(kd, m * kd * a, e)
        y.append((t - inv_alpha_cm(m) + (2.0 / 3.0) * 1j * kd ** 3) / kd ** 2)
    y = np.asarray(y)
    V = np.vander(np.asarray(kds) ** 2, 3, increasing=True)
    c, *_ = np.linalg.lstsq(V, y.real, rcond=None)
    return c[0], float(np.sum((a * e) ** 2).real), y


CASES = [(1.5, (0, 0, 1), (1, 0, 0)), (2.0, (0, 0, 1), (1, 0, 0)),
         (1.5, (1, 1, 0), (1, -1, 0)), (1.3, (1, 1, 1), (1, -1, 0)),
         (1.8, (1, 2, 2), (2, -2, 1)), (1.7, (0, 1, 0), (0, 0, 1))]


def test_ewald_sum_is_independent_of_the_split_parameter():
    vals = [lattice_sum(0.05, (0.0, 0.0, 0.075), (1.0, 0.0, 0.0), eta=eta)
            for eta in (1.5, SQPI, 2.2)]
    assert max(abs(v - vals[1]) for v in vals) < 1e-12 * abs(vals[1])


def test_lattice_sum_static_limit_is_clausius_mossotti():
    """kd -> 0 with |k| = m kd: the g = 0 term gives 4 pi/(m^2 - 1), the rest
    the Lorentz cavity field 4 pi/3; together 1/alpha_CM."""
    for m in (1.2, 1.5, 2.0):
        t = lattice_sum(1e-4, (0.0, 0.0, m * 1e-4), (0.0, 1.0, 0.0))
        assert abs(t - inv_alpha_cm(m)) < 1e-6


def test_lattice_sum_imaginary_part_is_radiative_reaction():
    """For |k| > kd the mode does not radiate: Im sum_{r != 0} = -(2/3) kd^3
    exactly (the r = 0 term of Im G is missing from a sum that vanishes)."""
    for kd in (0.02, 0.1, 0.3):
        t = lattice_sum(kd, (0.0, 1.5 * kd, 0.0), (1.0, 0.0, 0.0))
        assert abs(t.imag + (2.0 / 3.0) * kd ** 3) < 1e-12


def test_ldr_coefficients_from_lattice_dispersion_relation():
    with open(GOLDEN) as f:
        gold = json.load(f)
    assert (polarizability.LDR_B1, polarizability.LDR_B2, polarizability.LDR_B3) == \
        (gold["b1"], gold["b2"], gold["b3"])
    rows, rhs = [], []
    for m, a, e in CASES:
        c0, S, _ = kd2_coefficient(m, a, e)
        rows.append([1.0, m * m, S * m * m])
        rhs.append(c0)
    b, *_ = np.linalg.lstsq(np.asarray(rows), np.asarray(rhs), rcond=None)
    # the derivation reproduces all seven printed decimals
    assert abs(b[0] - polarizability.LDR_B1) < 1.5e-7, b
    assert abs(b[1] - polarizability.LDR_B2) < 1.5e-7, b
    assert abs(b[2] - polarizability.LDR_B3) < 1.5e-7, b
    # and the direction enters only through S: every case on the fitted plane
    resid = np.asarray(rows) @ b - np.asarray(rhs)
    assert np.max(np.abs(resid)) < 1e-7


def test_oracle_ldr_alpha_carries_the_lattice_wave():
    """The oracle's LDR alpha itself (not its constants) satisfies the
    dispersion relation to O(kd^4): 1/alpha - e.T.e shrinks like kd^4."""
    m = 1.6
    a = np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)     # S = 1/2: the b3 term counts
    e = np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0)
    err = []
    for kd in (0.02, 0.04):
        alpha = polarizability.alpha_diag(m, kd, "ldr", a, e)[0]
        err.append(abs(1.0 / alpha - lattice_sum(kd, m * kd * a, e)))
    assert err[0] < 1e-6
    assert err[1] / err[0] > 10.0          # ~16 for an O(kd^4) remainder
