"""Pins for the oracle's FFT product (O7/O8/O8b) and solvers (O9)."""
import numpy as np
import pytest

from oracle import dda, fft_matvec, lattice, polarizability, solvers, system
from paper_0704_0037_gb300 import inputs


def _problem(occ, m_list, kd, grid=None):
    return dda.Problem(occ, m_list, kd, grid)


def _beta(prob, presc="cldr", prop=(0.6, 0.0, 0.8), pol=(0.8, 0.0, -0.6)):
    return prob.beta(presc, prop, pol)


CASES = [
    ("sphere1", inputs.sphere(1)),
    ("sphere2", inputs.sphere(2)),
    ("sphere3", inputs.sphere(3)),
    ("sphere5", inputs.sphere(5)),
    ("sphere7", inputs.layered_sphere(7, 3)),
    ("cube3x5x7", inputs.cube(3, 5, 7)),
    ("ellipsoid12", inputs.ellipsoid(12, 9, 6)),
    ("random6x5x4", inputs.random_occupancy(6, 5, 4, 0.6, seed=11, n_mat=2)),
    ("sphere16", inputs.sphere(16)),
]


@pytest.mark.parametrize("name,occ", CASES, ids=[c[0] for c in CASES])
def test_fft_matvec_equals_bruteforce(name, occ):
    n_mat = int(occ.max())
    m_list = [1.5, 1.2 + 0.05j, 2.0][:n_mat]
    prob = _problem(occ, m_list, 0.55)
    beta = _beta(prob)
    x = inputs.random_vectors(5, 1, prob.n_occ)[0]
    y_ref = system.matvec_bruteforce(prob.pos, beta, prob.kd, x)
    y = prob.matvec(beta, "fft")(x)
    err = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    assert err < 1e-13, err


@pytest.mark.parametrize("rule", ["2n-1", "2n", "smooth+"])
def test_padding_rule(rule):
    """O8: any M >= 2n - 1 gives the same linear convolution."""
    occ = inputs.ellipsoid(7, 6, 5)
    nx, ny, nz = 7, 6, 5
    grid = {"2n-1": (2 * nx - 1, 2 * ny - 1, 2 * nz - 1),
            "2n": (2 * nx, 2 * ny, 2 * nz),
            "smooth+": (16, 15, 12)}[rule]
    prob = _problem(occ, [1.4], 0.5, grid)
    beta = _beta(prob)
    x = inputs.random_vectors(6, 1, prob.n_occ)[0]
    y_ref = system.matvec_bruteforce(prob.pos, beta, prob.kd, x)
    y = prob.matvec(beta, "fft")(x)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-13


def test_too_small_grid_rejected():
    with pytest.raises(ValueError):
        fft_matvec.dmatrix_full((4, 4, 4), (6, 8, 8), 0.5)


def test_octant_parity_rule():
    """O8b: D_mu,nu(.., M_a - k_a, ..) = (-1)^[odd along a] D_mu,nu(.., k_a, ..),
    odd along a iff exactly one of mu, nu equals a."""
    shape_n, shape_m = (5, 4, 3), (10, 9, 6)
    d = fft_matvec.dmatrix_full(shape_n, shape_m, 0.6)
    comps = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for c, (mu, nu) in enumerate(comps):
        for axis in range(3):                      # axis 0=x, 1=y, 2=z
            arr_axis = 3 - axis - 1 + 0            # array dims (z, y, x)
            odd = (mu == axis) != (nu == axis)
            flipped = np.roll(np.flip(d[c], axis=arr_axis), 1, axis=arr_axis)
            sign = -1.0 if odd else 1.0
            assert np.allclose(flipped, sign * d[c], rtol=1e-12, atol=1e-12 * np.abs(d[c]).max())


def test_conjugate_product_is_hermitian_adjoint():
    occ = inputs.sphere(5)
    prob = _problem(occ, [1.3 + 0.2j], 0.5)
    beta = _beta(prob)
    a = system.dense_matrix(prob.pos, beta, prob.kd)
    x = inputs.random_vectors(7, 1, prob.n_occ)[0]
    y = fft_matvec.matvec_fft(prob.occ, beta, prob.dmat(), x, conj=True)
    ref = (a.conj().T @ x.reshape(-1)).reshape(3, -1)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-13


def test_smooth_size():
    assert fft_matvec.smooth_size(267) == 270
    assert fft_matvec.smooth_size(31) == 32
    assert fft_matvec.smooth_size(13) == 14
    assert fft_matvec.smooth_size(1071) == 1080


# ---------------------------------------------------------------- solvers

def _solver_problem(m=1.5, n=6, presc="ldr"):
    occ = inputs.sphere(n)
    prob = _problem(occ, [m], lattice.kd_volume_corrected(1.5, int((occ > 0).sum())))
    prop, pol = (0, 0, 1), (1, 0, 0)
    beta = prob.beta(presc, prop, pol)
    b = system.rhs(beta, prob.pos, prob.kd, prop, pol)
    x_exact = system.solve_dense(prob.pos, beta, prob.kd, b)
    return prob, beta, b, x_exact


@pytest.mark.parametrize("name", list(solvers.SOLVERS))
@pytest.mark.parametrize("m", [1.5, 2.0 + 0.5j])
def test_solvers_reach_dense_solution(name, m):
    prob, beta, b, x_exact = _solver_problem(m)
    mv = prob.matvec(beta, "brute")
    x, info = solvers.SOLVERS[name](mv, b, tol=1e-11, maxiter=2000)
    assert info["status"] == "ok", info["status"]
    assert info["rel_res_true"] < 1e-11
    err = np.linalg.norm(x - x_exact) / np.linalg.norm(x_exact)
    assert err < 1e-9, err


def test_qmr_recurrence_tracks_true_residual():
    prob, beta, b, _ = _solver_problem(1.8)
    mv = prob.matvec(beta, "brute")
    x, info = solvers.qmr_cs(mv, b, tol=1e-9, maxiter=2000)
    assert abs(info["rel_res_true"] - info["rel_res_recur"]) < 1e-11
    # recompute the residual history with explicit products at a few steps
    assert info["hist"][0] == 1.0 and info["hist"][-1] < 1e-9


def test_qmr_iterates_are_quasi_minimal():
    """QMR by its definition: after k steps x_k = V_k z, z minimising
    ||rho_1 e_1 - H z||_2, where A V_k = V_{k+1} H is the complex-symmetric
    Lanczos relation in a unit-Euclidean-norm basis.  The basis here comes
    from explicit Gram-Schmidt with the bilinear form against every earlier
    vector and a least-squares solve, independent of the solver's
    recurrences."""
    prob, beta, b, _ = _solver_problem(1.8)
    mv = prob.matvec(beta, "brute")
    kmax = 8
    rho1 = np.linalg.norm(b)
    V = [b / rho1]
    H = np.zeros((kmax + 1, kmax), dtype=np.complex128)
    for j in range(kmax):
        w = mv(V[j])
        for i in range(j + 1):
            h = np.sum(V[i] * w) / np.sum(V[i] * V[i])
            H[i, j] += h
            w = w - h * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V.append(w / H[j + 1, j])
    assert np.abs(np.triu(H[:kmax, :kmax], 2)).max() < 1e-10 * np.abs(H).max()   # tridiagonal
    for k in (1, 3, 8):
        rhs = np.zeros(k + 1, dtype=np.complex128)
        rhs[0] = rho1
        z = np.linalg.lstsq(H[:k + 1, :k], rhs, rcond=None)[0]
        xk = sum(V[j] * z[j] for j in range(k))
        xq, info = solvers.qmr_cs(mv, b, tol=0.0, maxiter=k)
        assert info["iters"] == k
        assert np.linalg.norm(xq - xk) / np.linalg.norm(xk) < 1e-10


def test_matvec_counts():
    prob, beta, b, _ = _solver_problem(1.5)
    mv = prob.matvec(beta, "brute")
    for name, per_iter in (("qmr_cs", 1), ("bicg_cs", 1)):
        _, info = solvers.SOLVERS[name](mv, b, tol=1e-8)
        assert info["matvecs"] == info["iters"] * per_iter
    _, info = solvers.cgnr(mv, b, tol=1e-8)
    assert info["matvecs"] == 2 * info["iters"]


def test_maxiter_reports_not_converged():
    prob, beta, b, _ = _solver_problem(2.0)
    mv = prob.matvec(beta, "brute")
    for name in solvers.SOLVERS:
        _, info = solvers.SOLVERS[name](mv, b, tol=1e-12, maxiter=2)
        assert info["status"] == "not_converged"
        assert info["iters"] == 2


def test_identity_system_converges_in_one_step():
    """A = I (a single dipole): every solver returns b after one iteration."""
    b = np.array([[1.0 + 2j], [0.5j], [-0.3]])
    for name in solvers.SOLVERS:
        x, info = solvers.SOLVERS[name](lambda v: v, b, tol=1e-12)
        assert np.allclose(x, b, rtol=1e-15) and info["iters"] == 1


def test_bilinear_breakdown_single_dipole_circular_polarisation():
    """One dipole (A = I) under circular polarisation along z: b^T b = 0, so
    QMR-CS and Bi-CG-CS break down at their first step (no look-ahead, Sec. 2);
    Bi-CGSTAB (Hermitian products) solves it, x = b."""
    e = np.array([1.0, 1j, 0.0]) / np.sqrt(2.0)
    b = (0.7 + 0.2j) * e.reshape(3, 1)
    ident = lambda v: v.copy()          # noqa: E731
    for name in ("qmr_cs", "bicg_cs"):
        _, info = solvers.SOLVERS[name](ident, b, tol=1e-10, maxiter=10)
        assert info["status"] == solvers.BREAKDOWN, (name, info)
    x, info = solvers.SOLVERS["bicgstab"](ident, b, tol=1e-10, maxiter=10)
    assert info["status"] == solvers.OK
    assert np.allclose(x, b, rtol=0, atol=1e-15)
