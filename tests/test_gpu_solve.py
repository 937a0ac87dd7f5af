"""GPU parity of the solvers (Sec. 2) and scattering quantities (Sec. 3.1)
against the oracle, on the x = 3, m = 1.5 sphere at 16^3 (2,176 dipoles)
and smaller lattices."""
import numpy as np
import pytest

from oracle import mie, observables, solvers, system
from paper_0704_0037_gb300 import inputs

from gpu_util import need_gpu, rel_l2, twin

pytestmark = pytest.mark.gpu

PROP = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
POLS = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


@pytest.fixture(scope="module")
def sphere16():
    torch, dda = need_gpu()
    occ = inputs.sphere(16)
    p, prob = twin(occ, [1.5], None, volume_x=3.0)
    dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
    exact = []
    for r in range(2):
        beta = prob.beta("ldr", PROP[r], POLS[r])
        b = system.rhs(beta, prob.pos, prob.kd, PROP[r], POLS[r])
        exact.append(beta * system.solve_dense(prob.pos, beta, prob.kd, b))
    yield p, prob, np.stack(exact)
    p.close()


def _solve(p, solver, prec, tol, maxiter=2000, inner_tol=1e-3, hist_len=0, inner_cap=0):
    torch, dda = need_gpu()
    P = torch.zeros((2, 3, p.n_occ), dtype=torch.complex128, device="cuda")
    st, info, hist = dda.dda_solve(p.h, dict(solver=dda.SOLVER[solver], pol=dda.DDA_LDR,
                                             prec=dda.PREC[prec], tol=tol, maxiter=maxiter,
                                             inner_tol=inner_tol, inner_cap=inner_cap),
                                   PROP, POLS, P, hist_len)
    return st, info, P, hist


@pytest.mark.parametrize("solver", ["qmr_cs", "bicg_cs", "bicgstab", "cgnr"])
def test_solvers_fp64_reach_exact_solution(sphere16, solver):
    p, prob, exact = sphere16
    st, info, P, _ = _solve(p, solver, "fp64", 1e-10, maxiter=5000)
    assert st == 0, info
    for r in range(2):
        assert info[r]["rel_res_true"] < 1e-10
    assert rel_l2(P.cpu().numpy(), exact) < 1e-8


@pytest.mark.parametrize("solver", ["qmr_cs", "bicgstab"])
def test_fp32_refined_reaches_fp64_tolerance(sphere16, solver):
    p, prob, exact = sphere16
    st, info, P, _ = _solve(p, solver, "fp32_refined", 1e-9, maxiter=5000, inner_tol=1e-3)
    assert st == 0, info
    for r in range(2):
        assert info[r]["rel_res_true"] < 1e-9
        assert info[r]["outer"] >= 2 and info[r]["matvecs_fp64"] == info[r]["outer"]
    assert rel_l2(P.cpu().numpy(), exact) < 1e-7


def test_fp32_inner_floor_is_left_to_refinement(sphere16):
    """An inner tolerance below the complex64 rounding floor: the inner
    solves stop on stagnation and the FP64 refinement still reaches tol."""
    p, prob, exact = sphere16
    st, info, P, _ = _solve(p, "qmr_cs", "fp32_refined", 1e-9, maxiter=3000, inner_tol=1e-11)
    assert st == 0, info
    for r in range(2):
        assert info[r]["rel_res_true"] < 1e-9
        assert info[r]["outer"] >= 2
        assert info[r]["iters"] < 1000
    assert rel_l2(P.cpu().numpy(), exact) < 1e-7


def test_qmr_history_matches_oracle(sphere16):
    """Same algorithm, same arithmetic (FP64): the residual histories agree."""
    p, prob, _ = sphere16
    st, info, P, hist = _solve(p, "qmr_cs", "fp64", 1e-8, hist_len=400)
    beta = prob.beta("ldr", PROP[0], POLS[0])
    b = system.rhs(beta, prob.pos, prob.kd, PROP[0], POLS[0])
    _, oinfo = solvers.qmr_cs(prob.matvec(beta, "fft"), b, tol=1e-8)
    assert abs(info[0]["iters"] - oinfo["iters"]) <= 1
    k = min(info[0]["iters"], oinfo["iters"]) + 1
    h_gpu, h_ora = hist[0][:k], oinfo["hist"][:k]
    # rounding-order differences (GPU FFT vs numpy) grow slowly through the
    # Lanczos process: tight agreement while the residual is above 1e-6,
    # within 20 % (log distance < 0.08) down to the 1e-8 tail
    hi = h_ora > 1e-6
    assert np.allclose(h_gpu[hi], h_ora[hi], rtol=1e-5, atol=0), (h_gpu[:8], h_ora[:8])
    assert np.max(np.abs(np.log10(h_gpu) - np.log10(h_ora))) < 0.08


def test_observables_match_oracle(sphere16):
    torch, dda = need_gpu()
    p, prob, exact = sphere16
    st, info, P, _ = _solve(p, "qmr_cs", "fp64", 1e-10)
    th = inputs.angles_deg(181)
    dirs = observables.plane_dirs(th)
    F, q = dda.dda_scatter(p.h, dda.DDA_LDR, P, PROP, POLS, dirs)
    xs = 3.0
    for r in range(2):
        beta = prob.beta("ldr", PROP[r], POLS[r])
        alpha = beta * beta
        e = system.incident_field(prob.pos, prob.kd, PROP[r], POLS[r])
        qext = observables.q_ext(exact[r], e, prob.kd, xs)
        qabs = observables.q_abs(exact[r], alpha, prob.kd, xs)
        assert abs(q[r, 0] - qext) <= 1e-6 * abs(qext)
        assert abs(q[r, 1] - qabs) <= 1e-9 * abs(qext)          # real m: Q_abs = 0
        Fo = observables.farfield(exact[r], prob.pos, prob.kd, dirs)
        assert rel_l2(F[r], Fo) < 1e-7
    s11 = dda.dda_mueller_plane(th, F[0], F[1])
    Fx = observables.farfield(exact[0], prob.pos, prob.kd, dirs)
    Fy = observables.farfield(exact[1], prob.pos, prob.kd, dirs)
    s11_o = observables.s11_plane(Fx, Fy, th)
    assert np.max(np.abs(s11 - s11_o) / s11_o) <= 1e-6
    # physics: the paper's accuracy regime for x < 10 (Sec. 4)
    qm = mie.efficiencies(xs, 1.5)[0]
    assert abs(0.5 * (q[0, 0] + q[1, 0]) / qm - 1) < 0.03
    assert np.max(np.abs(s11 - mie.s11(xs, 1.5, th)) / mie.s11(xs, 1.5, th)) < 0.4


def test_qsca_quadrature_matches_oracle(sphere16):
    torch, dda = need_gpu()
    p, prob, exact = sphere16
    st, info, P, _ = _solve(p, "qmr_cs", "fp64", 1e-10)
    dirs, w = observables.sphere_quadrature(24, 48)
    F, q = dda.dda_scatter(p.h, dda.DDA_LDR, P, PROP, POLS, dirs, w)
    for r in range(2):
        qs = observables.q_sca_quadrature(exact[r], prob.pos, prob.kd, 3.0, 24, 48)
        assert abs(q[r, 2] - qs) <= 1e-6 * qs
        # energy balance of the converged DDA solution
        assert abs(q[r, 0] - q[r, 1] - q[r, 2]) <= 1e-5 * q[r, 0]


def test_mueller_full_and_single_polarisation_symmetry(sphere16):
    """All 16 in-plane Mueller elements against the oracle (exact solutions);
    the single-polarisation route (x-polarised solution + the 90 degree
    rotation symmetry of the sphere lattice, Sec. 3.1) gives the same matrix."""
    torch, dda = need_gpu()
    p, prob, exact = sphere16
    st, info, P, _ = _solve(p, "qmr_cs", "fp64", 1e-10)
    th = inputs.angles_deg(91)
    dirs = observables.plane_dirs(th)
    F, _ = dda.dda_scatter(p.h, dda.DDA_LDR, P, PROP, POLS, dirs)
    M = dda.dda_mueller_plane_full(th, F[0], F[1])
    Fo = [observables.farfield(exact[r], prob.pos, prob.kd, dirs) for r in range(2)]
    Mo = observables.mueller_plane(Fo[0], Fo[1], th)
    assert np.abs(M - Mo).max() <= 1e-7 * np.abs(Mo).max()
    assert dda.dda_symmetry(p.h) == dda.DDA_SYM_ROT90_Z
    Ms, Fx, Fy = dda.dda_mueller_plane_sym(p.h, dda.DDA_LDR, P[0], th)
    assert np.abs(Fx - F[0]).max() <= 1e-12 * np.abs(F[0]).max()
    assert np.abs(Ms - M).max() <= 1e-7 * np.abs(M).max()     # the two solves differ by ~tol
    # the cross-polarised elements vanish in this symmetry plane
    for (i, j) in ((0, 2), (0, 3), (2, 0), (3, 0), (1, 2), (1, 3)):
        assert np.abs(M[:, i, j]).max() <= 1e-8 * M[:, 0, 0].max()


def test_symmetry_flag_and_refusal():
    torch, dda = need_gpu()
    occ = inputs.ellipsoid(10, 8, 6)
    p, prob = twin(occ, [1.5], 0.5)
    with p:
        assert dda.dda_symmetry(p.h) == 0
        P = torch.zeros((3, p.n_occ), dtype=torch.complex128, device="cuda")
        with pytest.raises(dda.DDAError) as ei:
            dda.dda_mueller_plane_sym(p.h, dda.DDA_LDR, P, [0.0, 90.0])
        assert ei.value.status == dda.DDA_ERR_ARG
    # a cube with two materials arranged without the rotation symmetry
    occ = inputs.cube(6, 6, 4)
    occ[:, :, :3] = 2
    p, prob = twin(occ, [1.5, 1.3], 0.5)
    with p:
        assert dda.dda_symmetry(p.h) == 0
    occ = inputs.cube(6, 6, 4)
    p, prob = twin(occ, [1.5], 0.5)
    with p:
        assert dda.dda_symmetry(p.h) == dda.DDA_SYM_ROT90_Z


def test_asymmetry_parameter(sphere16):
    """<cos theta> from the library's amplitudes on a sphere quadrature against
    the oracle's, and against Mie within the paper's regime (Sec. 4)."""
    torch, dda = need_gpu()
    p, prob, exact = sphere16
    st, info, P, _ = _solve(p, "qmr_cs", "fp64", 1e-10)
    dirs, w = observables.sphere_quadrature(32, 64)
    F, q = dda.dda_scatter(p.h, dda.DDA_LDR, P, PROP, POLS, dirs, w)
    for r in range(2):
        g, gv = dda.dda_asymmetry(dirs, w, F[r], PROP[r])
        Fo = observables.farfield(exact[r], prob.pos, prob.kd, dirs)
        go, gvo = observables.asymmetry_from_farfield(Fo, dirs, w, PROP[r])
        assert abs(g - go) <= 1e-7 * abs(go)
        assert np.abs(gv[:2]).max() < 1e-6
        gm = mie.efficiencies(3.0, 1.5)[3]
        assert abs(g / gm - 1) < 0.03


def test_status_codes_and_edge_cases():
    torch, dda = need_gpu()
    occ = inputs.sphere(6)
    p, prob = twin(occ, [2.0], 0.6)
    with p:
        P = torch.zeros((1, 3, p.n_occ), dtype=torch.complex128, device="cuda")
        # solve before the D-matrix exists
        with pytest.raises(dda.DDAError) as ei:
            dda.dda_solve(p.h, dict(), PROP[:1], POLS[:1], P)
        assert ei.value.status == dda.DDA_ERR_STATE
        x = torch.zeros((1, 3, p.n_occ), dtype=torch.complex128, device="cuda")
        with pytest.raises(dda.DDAError):
            dda.dda_matvec(p.h, dda.DDA_FP64, x, torch.empty_like(x))
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP64)
        # maxiter = 1: not converged, still a valid iterate
        st, info, _ = dda.dda_solve(p.h, dict(tol=1e-12, maxiter=1), PROP[:1], POLS[:1], P)
        assert st == dda.DDA_NOT_CONVERGED and info[0]["iters"] == 1
        # FP32 mode without the FP32 D-matrix
        with pytest.raises(dda.DDAError) as ei:
            dda.dda_solve(p.h, dict(prec=dda.DDA_FP32_REFINED), PROP[:1], POLS[:1], P)
        assert ei.value.status == dda.DDA_ERR_STATE
        # bad arguments
        with pytest.raises(dda.DDAError) as ei:
            dda.dda_solve(p.h, dict(tol=-1.0), PROP[:1], POLS[:1], P)
        assert ei.value.status == dda.DDA_ERR_ARG
        with pytest.raises(dda.DDAError):
            dda.dda_set_beta(p.h, dda.DDA_LDR, [(np.nan, 0, 1)], [(1, 0, 0)])


def test_single_dipole_closed_form():
    torch, dda = need_gpu()
    occ = inputs.sphere(1)
    p, prob = twin(occ, [1.5], 0.4)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP64)
        P = torch.zeros((1, 3, 1), dtype=torch.complex128, device="cuda")
        st, info, _ = dda.dda_solve(p.h, dict(tol=1e-12), PROP[:1], POLS[:1], P)
        assert st == 0 and info[0]["iters"] == 1
        alpha = prob.alpha("ldr", PROP[0], POLS[0])[:, 0]
        assert np.allclose(P.cpu().numpy()[0, :, 0], alpha * POLS[0], rtol=1e-14, atol=1e-16)


def test_solve_is_deterministic(sphere16):
    p, prob, _ = sphere16
    _, i1, P1, h1 = _solve(p, "qmr_cs", "fp32_refined", 1e-6, hist_len=200)
    _, i2, P2, h2 = _solve(p, "qmr_cs", "fp32_refined", 1e-6, hist_len=200)
    assert np.array_equal(h1, h2)
    assert bool((P1 == P2).all())


def test_fp32_refined_switches_to_mixed_inner_solves(sphere16):
    """Inner solves with complex64 Krylov vectors are capped per refinement
    step; past the cap the next inner solves keep complex128 vectors with
    double-float products.  A cap of 5 steps forces the switch here; the
    solve still reaches the FP64 tolerance and the exact solution."""
    torch, dda = need_gpu()
    p, prob, exact = sphere16
    st, info, P, _ = _solve(p, "qmr_cs", "fp32_refined", 1e-9, maxiter=3000, inner_tol=1e-10,
                            inner_cap=5)
    assert st == 0, info
    for r in range(2):
        assert info[r]["rel_res_true"] < 1e-9
        assert info[r]["outer"] >= 2
    assert rel_l2(P.cpu().numpy(), exact) < 1e-7


@pytest.mark.parametrize("prec_name", ["fp64", "fp32_refined"])
def test_residual_entry_point_against_oracle(sphere16, prec_name):
    """dda_residual recomputes ||b - A x|| / ||b|| with the FP64 product from P
    alone; it agrees with the oracle's residual of the same P (its own FFT
    product, x = P / beta) and with the solver's exit value."""
    torch, dda = need_gpu()
    p, prob, exact = sphere16
    st, info, P, _ = _solve(p, "qmr_cs", prec_name, 1e-5, maxiter=500, inner_tol=1e-3)
    assert st == 0, info
    res = dda.dda_residual(p.h, dda.DDA_LDR, P, PROP, POLS)
    Pn = P.cpu().numpy()
    for r in range(2):
        beta = prob.beta("ldr", PROP[r], POLS[r])
        b = system.rhs(beta, prob.pos, prob.kd, PROP[r], POLS[r])
        x = Pn[r] / beta
        ref = np.linalg.norm(b - prob.matvec(beta, "fft")(x)) / np.linalg.norm(b)
        assert abs(res[r] - ref) <= 1e-6 * ref, (res[r], ref)
        assert abs(res[r] - info[r]["rel_res_true"]) <= 1e-3 * ref
        assert res[r] < 1e-5
    # the exact (dense) solution has a residual at the rounding level
    Pe = torch.from_numpy(exact).cuda()
    res_e = dda.dda_residual(p.h, dda.DDA_LDR, Pe, PROP, POLS)
    assert np.all(res_e < 1e-12)
