"""Pins for the Green's tensor (O4), polarizabilities (O3) and the system (O5/O6)."""
import math

import numpy as np
import pytest

from oracle import green, lattice, polarizability, system


def test_green_symmetry():
    rng = np.random.default_rng(1)
    d = rng.standard_normal((50, 3)) * 3
    g = green.green_tensor(d, 0.7)
    assert np.allclose(g, np.swapaxes(g, -1, -2), rtol=0, atol=0)
    assert np.allclose(green.green_tensor(-d, 0.7), g, rtol=0, atol=1e-15)
    assert np.all(green.green_tensor(np.zeros((1, 3)), 0.7) == 0)


def test_green_static_limit():
    rng = np.random.default_rng(2)
    d = rng.standard_normal((20, 3)) * 2 + 0.5
    g = green.green_tensor(d, 1e-7)
    s = green.green_static(d)
    assert np.allclose(g, s, rtol=1e-10, atol=1e-12)


def test_green_is_hessian_of_scalar_green():
    """Independent form: G = (kappa^2 I + grad grad) exp(i kappa r)/r, with the
    Hessian taken numerically to high precision by mpmath."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    kd = 0.9
    r0 = [1.3, -0.7, 2.1]

    def phi(x, y, z):
        r = mpmath.sqrt(x * x + y * y + z * z)
        return mpmath.exp(1j * kd * r) / r

    g = green.green_tensor(np.array(r0), kd)
    for mu in range(3):
        for nu in range(3):
            order = [0, 0, 0]
            order[mu] += 1
            order[nu] += 1
            h = complex(mpmath.diff(phi, tuple(r0), tuple(order)))
            ref = h + (kd * kd * complex(phi(*r0)) if mu == nu else 0.0)
            assert abs(g[mu, nu] - ref) < 1e-13 * abs(g).max()


def test_alpha_cm_closed_form():
    a = polarizability.alpha_cm(1.5)
    assert abs(a - 3 / (4 * math.pi) * 1.25 / 4.25) < 1e-16
    assert polarizability.alpha_cm(1.0) == 0


@pytest.mark.parametrize("presc", ["rr", "ldr", "cldr"])
def test_radiative_reaction_exact_for_real_m(presc):
    """Im(1/alpha) = -(2/3) kappa^3 exactly for real m (so Q_abs vanishes)."""
    for m in (1.05, 1.5, 2.0):
        for kd in (0.1, 0.37, 0.6):
            a = polarizability.alpha_diag(m, kd, presc, prop=(0.6, 0, 0.8), pol=(0.8, 0, -0.6))
            assert np.allclose(np.imag(1 / a), -(2 / 3) * kd ** 3, rtol=1e-12, atol=0)


@pytest.mark.parametrize("presc", ["rr", "ldr", "cldr"])
def test_small_kd_limit_is_cm(presc):
    a = polarizability.alpha_diag(1.7 + 0.2j, 1e-6, presc)
    assert np.allclose(a, polarizability.alpha_cm(1.7 + 0.2j), rtol=1e-10)


def test_ldr_s_term_and_cldr():
    m, kd = 1.5, 0.4
    # S = 0 for incidence along z with x or y polarisation: both equal
    ax = polarizability.alpha_diag(m, kd, "ldr", (0, 0, 1), (1, 0, 0))
    ay = polarizability.alpha_diag(m, kd, "ldr", (0, 0, 1), (0, 1, 0))
    assert np.array_equal(ax, ay)
    # S = sum (a_mu e_mu)^2 enters with b3 m^2 kappa^2
    a, e = np.array([1, 1, 0]) / math.sqrt(2), np.array([1, -1, 0]) / math.sqrt(2)
    s = np.sum((a * e) ** 2)
    ref = 1 / polarizability.alpha_cm(m) + (polarizability.LDR_B1 + polarizability.LDR_B2 * m * m
                                            + polarizability.LDR_B3 * s * m * m) * kd ** 2 \
        - 2j / 3 * kd ** 3
    assert np.allclose(polarizability.alpha_diag(m, kd, "ldr", a, e), 1 / ref, rtol=1e-14)
    # CLDR along z: xx, yy components coincide with LDR at S = 0; zz differs
    c = polarizability.alpha_diag(m, kd, "cldr", (0, 0, 1), (1, 0, 0))
    assert np.allclose(c[:2], ax[:2], rtol=1e-15)
    assert abs(c[2] - ax[2]) > 1e-4


def test_beta_is_principal_sqrt():
    b = polarizability.beta_diag(1.3 + 0.4j, 0.5, "ldr")
    assert np.allclose(b * b, polarizability.alpha_diag(1.3 + 0.4j, 0.5, "ldr"), rtol=1e-15)
    assert np.all(np.real(b) >= 0)


def _small_problem(n=4, m=(1.5,), seed=0):
    occ = lattice.sphere_occupancy(n) if n > 2 else lattice.cube_occupancy(n, n, n)
    pos = lattice.positions(occ)
    rng = np.random.default_rng(seed)
    mat = rng.integers(0, len(m), size=pos.shape[0])
    kd = 0.45
    tab = np.stack([polarizability.beta_diag(mm, kd, "cldr", (0.6, 0, 0.8)) for mm in m])
    beta = polarizability.per_dipole(tab, mat)
    return pos, beta, kd


def test_dense_matrix_is_complex_symmetric():
    pos, beta, kd = _small_problem(5, m=(1.5, 1.2 + 0.1j))
    a = system.dense_matrix(pos, beta, kd)
    # complex symmetric up to rounding of the beta_i beta_j products
    assert np.abs(a - a.T).max() <= 1e-15 * np.abs(a).max()
    assert np.abs(a - a.conj().T).max() > 1e-3      # but not Hermitian
    n = pos.shape[0]
    assert np.allclose(np.diag(a), 1.0)
    # off-diagonal blocks are -beta_i G_ij beta_j
    i, j = 3, 7
    g = green.green_tensor(pos[i] - pos[j], kd)
    blk = np.array([[a[mu * n + i, nu * n + j] for nu in range(3)] for mu in range(3)])
    assert np.allclose(blk, -beta[:, i][:, None] * g * beta[:, j][None, :], rtol=1e-15)


def test_bruteforce_matches_dense():
    pos, beta, kd = _small_problem(6, m=(1.5, 2.0 + 0.3j))
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, pos.shape[0])) + 1j * rng.standard_normal((3, pos.shape[0]))
    a = system.dense_matrix(pos, beta, kd)
    y1 = (a @ x.reshape(-1)).reshape(3, -1)
    y2 = system.matvec_bruteforce(pos, beta, kd, x, chunk=17)
    assert np.linalg.norm(y1 - y2) / np.linalg.norm(y1) < 1e-13


def test_sampled_rows_match_dense():
    """The chunked per-output direct sum (for sampled outputs of large
    lattices) equals rows of the dense Eq. (2) matrix, chunk edges included."""
    pos, beta, kd = _small_problem(6, m=(1.5, 2.0 + 0.3j))
    n = pos.shape[0]
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    a = system.dense_matrix(pos, beta, kd)
    y = (a @ x.reshape(-1)).reshape(3, -1)
    rows = [0, n - 1, n // 2, 5]
    for chunk in (7, n, 1 << 21):
        ys = system.matvec_rows(pos, beta, kd, x, rows, chunk=chunk)
        assert np.abs(ys - y[:, rows]).max() <= 1e-13 * np.abs(y).max()


def test_single_dipole_closed_form():
    """N = 1: A = I, so x = b and P = alpha E_inc."""
    pos = np.zeros((1, 3))
    kd = 0.3
    alpha = polarizability.alpha_diag(1.5, kd, "ldr")
    beta = np.sqrt(alpha)[:, None]
    b = system.rhs(beta, pos, kd, (0, 0, 1), (1, 0, 0))
    x = system.solve_dense(pos, beta, kd, b)
    assert np.allclose(beta * x, alpha[:, None] * np.array([[1], [0], [0]]), rtol=1e-15)
