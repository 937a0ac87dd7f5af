"""Checkpoint and resume of a QMR-CS solve (ADDA saves its iterative
solver's state so that a long run can be stopped and continued, Sec. 2).

The library writes the state into a host buffer the caller owns.  A solve
of 2k iterations and a solve stopped after k iterations, then resumed from
its image for the rest, must give the same polarizations bit for bit, in
FP64 (state saved at a host synchronisation) and in the FP32-refined form
(state saved between refinement steps).
"""
import numpy as np
import pytest

from paper_0704_0037_gb300 import inputs

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

PROP = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
POLS = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


@pytest.fixture(scope="module")
def sphere():
    torch, dda = need_gpu()
    occ = inputs.sphere(18)
    p = dda.Particle(occ, [2.0], 5.0, volume_corrected=True)
    dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
    yield p
    p.close()


def _solve(p, prec, **kw):
    torch, dda = need_gpu()
    P = torch.zeros((2, 3, p.n_occ), dtype=torch.complex128, device="cuda")
    opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_LDR, prec=prec, tol=1e-16, maxiter=48,
                inner_tol=1e-3)
    opts.update(kw)
    st, info, _ = dda.dda_solve(p.h, opts, PROP, POLS, P)
    return st, info, P


def test_fp64_stop_and_resume_is_bit_identical(sphere):
    torch, dda = need_gpu()
    p = sphere
    nbytes = dda.dda_checkpoint_bytes(p.h, dda.DDA_FP64, 2)
    assert nbytes > 8 * 2 * 3 * p.n_occ * 16
    st_a, info_a, P_a = _solve(p, dda.DDA_FP64)
    assert st_a == dda.DDA_NOT_CONVERGED and info_a[0]["iters"] == 48
    buf = np.zeros(nbytes, dtype=np.uint8)
    st_b, info_b, P_b = _solve(p, dda.DDA_FP64, checkpoint_every=24, checkpoint=buf,
                               checkpoint_stop=True)
    assert st_b == dda.DDA_NOT_CONVERGED and info_b[0]["iters"] == 24
    assert not torch.equal(P_b, P_a)
    st_c, info_c, P_c = _solve(p, dda.DDA_FP64, checkpoint=buf, resume=True)
    assert info_c[0]["iters"] == 48 and info_c[1]["iters"] == 48
    assert torch.equal(P_c, P_a)
    for r in range(2):
        assert info_c[r]["rel_res_true"] == info_a[r]["rel_res_true"]


def test_fp64_checkpoint_without_stop_leaves_the_solve_unchanged(sphere):
    torch, dda = need_gpu()
    p = sphere
    buf = np.zeros(dda.dda_checkpoint_bytes(p.h, dda.DDA_FP64, 2), dtype=np.uint8)
    _, _, P_a = _solve(p, dda.DDA_FP64, maxiter=40)
    _, info_b, P_b = _solve(p, dda.DDA_FP64, maxiter=40, checkpoint_every=16, checkpoint=buf)
    assert torch.equal(P_b, P_a) and info_b[0]["iters"] == 40
    # the image holds the state after 32 steps: resuming it repeats the last 8
    _, info_c, P_c = _solve(p, dda.DDA_FP64, maxiter=40, checkpoint=buf, resume=True)
    assert torch.equal(P_c, P_a) and info_c[0]["iters"] == 40


def test_fp32_refined_stop_and_resume_is_bit_identical(sphere):
    torch, dda = need_gpu()
    p = sphere
    kw = dict(tol=1e-9, maxiter=4000, inner_tol=1e-3)
    st_a, info_a, P_a = _solve(p, dda.DDA_FP32_REFINED, **kw)
    assert st_a == dda.DDA_OK and info_a[0]["outer"] >= 3, info_a
    buf = np.zeros(dda.dda_checkpoint_bytes(p.h, dda.DDA_FP32_REFINED, 2), dtype=np.uint8)
    st_b, info_b, P_b = _solve(p, dda.DDA_FP32_REFINED, checkpoint_every=1, checkpoint=buf,
                               checkpoint_stop=True, **kw)
    assert st_b == dda.DDA_NOT_CONVERGED and info_b[0]["outer"] == 1, info_b
    st_c, info_c, P_c = _solve(p, dda.DDA_FP32_REFINED, checkpoint=buf, resume=True, **kw)
    assert st_c == dda.DDA_OK
    assert torch.equal(P_c, P_a)
    for r in range(2):
        for k in ("iters", "outer", "matvecs", "rel_res_true"):
            assert info_c[r][k] == info_a[r][k], (k, info_c[r], info_a[r])


def test_resume_refuses_another_incidence_or_a_short_buffer(sphere):
    torch, dda = need_gpu()
    p = sphere
    buf = np.zeros(dda.dda_checkpoint_bytes(p.h, dda.DDA_FP64, 2), dtype=np.uint8)
    _solve(p, dda.DDA_FP64, checkpoint_every=8, checkpoint=buf, checkpoint_stop=True)
    P = torch.zeros((2, 3, p.n_occ), dtype=torch.complex128, device="cuda")
    opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_LDR, prec=dda.DDA_FP64, tol=1e-16, maxiter=48,
                checkpoint=buf, resume=True)
    with pytest.raises(dda.DDAError) as ei:
        dda.dda_solve(p.h, opts, PROP, POLS[::-1].copy(), P)
    assert ei.value.status == dda.DDA_ERR_ARG
    with pytest.raises(dda.DDAError) as ei:
        dda.dda_solve(p.h, dict(opts, checkpoint=buf[:-1]), PROP, POLS, P)
    assert ei.value.status == dda.DDA_ERR_ARG
    # the per-right-hand-side path (a residual history) takes no checkpoints
    with pytest.raises(dda.DDAError) as ei:
        dda.dda_solve(p.h, dict(opts, resume=False, checkpoint_every=8), PROP, POLS, P, 8)
    assert ei.value.status == dda.DDA_ERR_ARG
