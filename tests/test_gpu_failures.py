"""Failure paths of the solvers and of the device-memory budget, reached from
host inputs (no GPU fault is provoked).

* Breakdown: one dipole has no interactions (G(0) = 0), so A = I and b is
  beta E_inc.  Under circular polarisation e = (1, i, 0)/sqrt(2) with
  incidence along z, b^T b = beta^2 (e . e) = 0: the bilinear form that QMR
  and Bi-CG use for a complex-symmetric A (Sec. 2) vanishes at the first
  step, a breakdown these solvers have without look-ahead.  Bi-CGSTAB uses
  the Hermitian product and solves it.
* Non-finite values: a refractive index of 1e155 is a finite double, but
  eps = m^2 overflows, so alpha and beta are NaN and the first reduction of
  every solver sees it.
* Out of memory: a cap on the library's device memory makes the D-matrix
  build fail as an exhausted device would; the handle stays usable and the
  build succeeds once the cap is lifted.
"""
import numpy as np
import pytest

from paper_0704_0037_gb300 import inputs

from gpu_util import need_gpu, rel_l2

pytestmark = pytest.mark.gpu

CIRC = [[1 / np.sqrt(2), 1j / np.sqrt(2), 0.0]]
LIN = [[1.0, 0.0, 0.0]]
ZDIR = [[0.0, 0.0, 1.0]]


def _opts(dda, solver, prec, **kw):
    o = dict(solver=solver, pol=dda.DDA_LDR, prec=prec, tol=1e-8, maxiter=50, inner_tol=1e-3)
    o.update(kw)
    return o


@pytest.mark.parametrize("prec_name", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("solver_name,hist", [("qmr_cs", 0), ("qmr_cs", 8), ("bicg_cs", 0)])
def test_single_dipole_circular_polarisation_breaks_down(prec_name, solver_name, hist):
    torch, dda = need_gpu()
    occ = np.ones((1, 1, 1), dtype=np.uint8)
    with dda.Particle(occ, [1.5], 0.4) as p:
        prec = dda.PREC[prec_name]
        dda.dda_build_Dmatrix(p.h, prec)
        P = torch.zeros((1, 3, 1), dtype=torch.complex128, device="cuda")
        st, info, _ = dda.dda_solve(p.h, _opts(dda, dda.SOLVER[solver_name], prec), ZDIR, CIRC,
                                    P, hist)
        assert st == dda.DDA_BREAKDOWN, info
        assert info[0]["status"] == dda.DDA_BREAKDOWN
        # the handle stays usable: linear polarisation solves at once (A = I)
        st, info, _ = dda.dda_solve(p.h, _opts(dda, dda.SOLVER[solver_name], prec), ZDIR, LIN,
                                    P, hist)
        assert st == dda.DDA_OK, info
        from oracle import polarizability
        alpha = polarizability.alpha_diag(1.5, p.kd, "ldr", ZDIR[0], LIN[0])
        assert abs(P[0, 0, 0].item() - alpha[0]) <= 1e-12 * abs(alpha[0])


def test_single_dipole_circular_polarisation_bicgstab_solves():
    """Bi-CGSTAB's Hermitian products do not vanish: the same right-hand side
    is solved, P = alpha E."""
    torch, dda = need_gpu()
    occ = np.ones((1, 1, 1), dtype=np.uint8)
    with dda.Particle(occ, [1.5], 0.4) as p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP64)
        P = torch.zeros((1, 3, 1), dtype=torch.complex128, device="cuda")
        st, info, _ = dda.dda_solve(p.h, _opts(dda, dda.DDA_BICGSTAB, dda.DDA_FP64), ZDIR, CIRC, P)
        assert st == dda.DDA_OK, info
        from oracle import polarizability
        alpha = polarizability.alpha_diag(1.5, p.kd, "ldr", ZDIR[0], CIRC[0])
        ref = alpha * np.asarray(CIRC[0])
        assert rel_l2(P[0, :, 0].cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("prec_name", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("solver_name,hist", [("qmr_cs", 0), ("qmr_cs", 8), ("bicgstab", 0),
                                              ("cgnr", 0)])
def test_overflowing_refractive_index_is_nonfinite(prec_name, solver_name, hist):
    torch, dda = need_gpu()
    occ = inputs.sphere(6)
    with dda.Particle(occ, [1e155], 0.3) as p:
        prec = dda.PREC[prec_name]
        dda.dda_build_Dmatrix(p.h, prec)
        P = torch.zeros((1, 3, p.n_occ), dtype=torch.complex128, device="cuda")
        with pytest.raises(dda.DDAError) as ei:
            dda.dda_solve(p.h, _opts(dda, dda.SOLVER[solver_name], prec), ZDIR, LIN, P, hist)
        assert ei.value.status == dda.DDA_ERR_NONFINITE


def test_memory_cap_gives_oom_and_the_handle_recovers():
    torch, dda = need_gpu()
    occ = inputs.sphere(20)
    dda.dda_release_cached_memory()
    live0, _ = dda.dda_memory_in_use()
    try:
        with dda.Particle(occ, [1.3], 0.5) as p:
            live1, _ = dda.dda_memory_in_use()
            assert live1 > live0                          # the lattice arrays
            dda.dda_set_memory_limit(live1 + 4096)        # far below a D-matrix
            with pytest.raises(dda.DDAError) as ei:
                dda.dda_build_Dmatrix(p.h, dda.DDA_FP64)
            assert ei.value.status == dda.DDA_ERR_OOM
            dda.dda_set_memory_limit(0)
            dda.dda_build_Dmatrix(p.h, dda.DDA_FP64)
            dda.dda_set_beta(p.h, dda.DDA_LDR, ZDIR, LIN)
            x = torch.from_numpy(inputs.random_vectors(3, 1, p.n_occ)).cuda()
            y = torch.empty_like(x)
            dda.dda_matvec(p.h, dda.DDA_FP64, x, y)
            from gpu_util import twin
            q, prob = twin(occ, [1.3], 0.5)
            q.close()
            beta = prob.beta("ldr", ZDIR[0], LIN[0])
            ref = prob.matvec(beta, "fft")(x.cpu().numpy()[0])
            assert rel_l2(y.cpu().numpy()[0], ref) <= 1e-12
    finally:
        dda.dda_set_memory_limit(0)
    live2, _ = dda.dda_memory_in_use()
    assert live2 == live0
