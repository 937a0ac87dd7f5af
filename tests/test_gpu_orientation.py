"""GPU parity of orientation averaging (Sec. 2: Euler angles, alpha by
scattering planes, beta and gamma by independent solutions) against the
oracle's restatement, on an asymmetric two-material particle."""
import numpy as np
import pytest

from oracle import dda as odda
from oracle import orientation, system
from paper_0704_0037_gb300 import inputs

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_orientation_average_matches_oracle():
    torch, dda = need_gpu()
    occ = inputs.ellipsoid(7, 5, 4)
    occ[:, :, :3] *= 2
    m = [1.5 + 0.05j, 1.3]
    kd = 0.5
    th = np.arange(0.0, 181.0, 10.0)
    p = dda.Particle(occ, m, kd)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP64)
        opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_CLDR, prec=dda.DDA_FP64, tol=1e-11,
                    maxiter=2000)
        st, q, M, infos = dda.dda_orientation_average(p.h, opts, 3, 2, 3, th)
        assert st == 0 and len(infos) == 12 and all(i["status"] == 0 for i in infos)
        prob = odda.Problem(occ, m, p.kd)
        solve = lambda beta, b: system.solve_dense(prob.pos, beta, prob.kd, b)   # noqa: E731
        x_size = p.kd * (3 * p.n_occ / (4 * np.pi)) ** (1 / 3)
        qe, qa, Mo = orientation.average(prob, x_size, "cldr", 3, 2, 3, th, solve)
        assert abs(q[0] - qe) <= 1e-8 * abs(qe) and abs(q[1] - qa) <= 1e-8 * abs(qe)
        assert np.abs(M - Mo).max() <= 1e-8 * np.abs(Mo).max()
        # the refinement form reaches the same averages to its tolerance
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        st, q32, M32, _ = dda.dda_orientation_average(
            p.h, dict(opts, prec=dda.DDA_FP32_REFINED, tol=1e-9, inner_tol=1e-4), 3, 2, 3, th)
        assert st == 0 and abs(q32[0] - qe) <= 1e-7 * abs(qe)
        assert np.abs(M32 - Mo).max() <= 1e-7 * np.abs(Mo).max()
        with pytest.raises(dda.DDAError) as ei:
            dda.dda_orientation_average(p.h, dict(opts, pol=dda.DDA_LDR), 3, 2, 3, th)
        assert ei.value.status == dda.DDA_ERR_ARG
