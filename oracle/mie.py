"""O11: Mie series for a homogeneous sphere (the exact reference of Sec. 3.1).

Sec. 3.1 compares every DDA result with the Mie theory for the same sphere.
The series is restated here from the mathematics (Riccati-Bessel functions
psi_n(z) = z j_n(z), chi_n(z) = -z y_n(z), xi_n = psi_n - i chi_n, the
logarithmic derivative D_n(z) = psi_n'(z)/psi_n(z)):

  a_n = [(D_n(mx)/m + n/x) psi_n(x) - psi_{n-1}(x)] / [(D_n(mx)/m + n/x) xi_n(x) - xi_{n-1}(x)]
  b_n = [(m D_n(mx) + n/x) psi_n(x) - psi_{n-1}(x)] / [(m D_n(mx) + n/x) xi_n(x) - xi_{n-1}(x)]
  Q_ext = (2/x^2) sum (2n+1) Re(a_n + b_n),   Q_sca = (2/x^2) sum (2n+1)(|a_n|^2 + |b_n|^2)
  S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),  S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n)
  S11 = (|S1|^2 + |S2|^2) / 2

psi_n, chi_n by upward recurrence f_{n+1} = (2n+1)/x f_n - f_{n-1}; D_n by
downward recurrence D_{n-1} = n/z - 1/(D_n + n/z) started well above
max(n_max, |m x|);
series truncated at n_max = x + 4 x^(1/3) + 2; angular functions by
pi_n = ((2n-1) mu pi_{n-1} - n pi_{n-2}) / (n-1), tau_n = n mu pi_n - (n+1) pi_{n-1}.
"""
import math

import numpy as np


def n_terms(x):
    return int(round(x + 4.0 * x ** (1.0 / 3.0) + 2.0))


def coefficients(x, m):
    """Mie coefficients a_n, b_n for n = 1..n_max (complex arrays)."""
    m = complex(m)
    nmax = n_terms(x)
    z = m * x
    # the downward recurrence forgets its (zero) start value only well above
    # |z|; start far enough up that the error at n <= n_max is at round-off
    nstart = int(1.2 * max(nmax, abs(z))) + 64
    D = np.zeros(nstart + 1, dtype=np.complex128)
    for n in range(nstart, 0, -1):
        D[n - 1] = n / z - 1.0 / (D[n] + n / z)
    psi = np.zeros(nmax + 1)
    chi = np.zeros(nmax + 1)
    psi_m1, chi_m1 = math.cos(x), -math.sin(x)
    psi[0], chi[0] = math.sin(x), math.cos(x)
    for n in range(1, nmax + 1):
        prev_psi = psi_m1 if n == 1 else psi[n - 2]
        prev_chi = chi_m1 if n == 1 else chi[n - 2]
        psi[n] = (2 * n - 1) / x * psi[n - 1] - prev_psi
        chi[n] = (2 * n - 1) / x * chi[n - 1] - prev_chi
    xi = psi - 1j * chi
    n = np.arange(1, nmax + 1)
    Dn = D[1:nmax + 1]
    ta = Dn / m + n / x
    tb = m * Dn + n / x
    a = (ta * psi[1:] - psi[:-1]) / (ta * xi[1:] - xi[:-1])
    b = (tb * psi[1:] - psi[:-1]) / (tb * xi[1:] - xi[:-1])
    return a, b


def efficiencies(x, m):
    """(Q_ext, Q_sca, Q_abs, g) of a sphere with size parameter x, index m."""
    a, b = coefficients(x, m)
    n = np.arange(1, a.size + 1)
    qext = 2.0 / x ** 2 * float(np.sum((2 * n + 1) * np.real(a + b)))
    qsca = 2.0 / x ** 2 * float(np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2)))
    an, bn = a[:-1], b[:-1]
    a1, b1 = a[1:], b[1:]
    nn = n[:-1]
    g1 = np.sum(nn * (nn + 2) / (nn + 1) * np.real(an * np.conj(a1) + bn * np.conj(b1)))
    g2 = np.sum((2 * n + 1) / (n * (n + 1)) * np.real(a * np.conj(b)))
    g = 4.0 / (x ** 2 * qsca) * float(g1 + g2) if qsca > 0 else 0.0
    return qext, qsca, qext - qsca, g


def amplitudes(x, m, thetas_deg):
    """S1(theta), S2(theta) for angles in degrees."""
    a, b = coefficients(x, m)
    nmax = a.size
    mu = np.cos(np.deg2rad(np.asarray(thetas_deg, dtype=np.float64)))
    S1 = np.zeros(mu.shape, dtype=np.complex128)
    S2 = np.zeros(mu.shape, dtype=np.complex128)
    pi_prev = np.zeros_like(mu)          # pi_0
    pi_cur = np.ones_like(mu)            # pi_1
    for n in range(1, nmax + 1):
        if n > 1:
            pi_new = ((2 * n - 1) * mu * pi_cur - n * pi_prev) / (n - 1)
            pi_prev, pi_cur = pi_cur, pi_new
        tau = n * mu * pi_cur - (n + 1) * pi_prev
        f = (2 * n + 1) / (n * (n + 1))
        S1 += f * (a[n - 1] * pi_cur + b[n - 1] * tau)
        S2 += f * (a[n - 1] * tau + b[n - 1] * pi_cur)
    return S1, S2


def s11(x, m, thetas_deg):
    S1, S2 = amplitudes(x, m, thetas_deg)
    return 0.5 * (np.abs(S1) ** 2 + np.abs(S2) ** 2)
