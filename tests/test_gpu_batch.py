"""Batched right-hand sides: one launch per product pass for all of them
(dda_matvec with nrhs > 1) and the batched QMR-CS (dda_solve_batch), against
the one-at-a-time path and the oracle's exact solutions."""
import numpy as np
import pytest

from oracle import system
from paper_0704_0037_gb300 import inputs

from gpu_util import need_gpu, rel_l2, twin

pytestmark = pytest.mark.gpu


def _orientations(k, seed):
    a = inputs.random_unit_vectors(seed, k)
    prop, pol = [], []
    for ai in a:
        for e in inputs.perpendicular_pols(ai):
            prop.append(ai)
            pol.append(e)
    return np.array(prop), np.array(pol)


@pytest.mark.parametrize("name,occ", [("sphere16", inputs.sphere(16)),
                                      ("ellipsoid13x9x7", inputs.ellipsoid(13, 9, 7))])
def test_batched_product_equals_single(name, occ):
    torch, dda = need_gpu()
    p, prob = twin(occ, [1.6 + 0.05j], 0.5)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        prop, pol = _orientations(3, 5)
        dda.dda_set_beta(p.h, dda.DDA_CLDR, prop, pol)
        for prec, dt in ((dda.DDA_FP64, torch.complex128), (dda.DDA_FP32_REFINED, torch.complex64)):
            x = torch.from_numpy(inputs.random_vectors(9, 6, p.n_occ)).to("cuda", dt)
            y = torch.empty_like(x)
            dda.dda_matvec(p.h, prec, x, y, nrhs=6)
            for r in range(6):
                dda.dda_set_beta(p.h, dda.DDA_CLDR, prop[r:r + 1], pol[r:r + 1])
                y1 = torch.empty_like(x[r:r + 1])
                dda.dda_matvec(p.h, prec, x[r:r + 1], y1)
                assert torch.equal(y1[0], y[r]), (name, prec, r)
            dda.dda_set_beta(p.h, dda.DDA_CLDR, prop, pol)
            if prec == dda.DDA_FP64:
                for r in (0, 5):
                    beta = prob.beta("cldr", prop[r], pol[r])
                    ref = prob.matvec(beta, "fft")(x[r].cpu().numpy())
                    assert rel_l2(y[r].cpu().numpy(), ref) < 1e-12


@pytest.fixture(scope="module")
def sphere16_cldr():
    torch, dda = need_gpu()
    occ = inputs.sphere(16)
    p, prob = twin(occ, [1.5 + 0.02j], None, volume_x=3.0)
    dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
    prop, pol = _orientations(4, 11)
    exact = []
    for r in range(len(prop)):
        beta = prob.beta("cldr", prop[r], pol[r])
        b = system.rhs(beta, prob.pos, prob.kd, prop[r], pol[r])
        exact.append(beta * system.solve_dense(prob.pos, beta, prob.kd, b))
    yield p, prob, prop, pol, np.stack(exact)
    p.close()


def test_solve_batch_fp64_equals_sequential(sphere16_cldr):
    torch, dda = need_gpu()
    p, prob, prop, pol, exact = sphere16_cldr
    opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_CLDR, prec=dda.DDA_FP64, tol=1e-10, maxiter=3000)
    Pb = torch.zeros((len(prop), 3, p.n_occ), dtype=torch.complex128, device="cuda")
    st, info = dda.dda_solve_batch(p.h, opts, prop, pol, Pb)
    assert st == 0
    Ps = torch.zeros_like(Pb)
    st2, info2, _ = dda.dda_solve(p.h, opts, prop, pol, Ps)
    for r in range(len(prop)):
        assert info[r]["status"] == 0 and info[r]["rel_res_true"] < 1e-10
        assert info[r]["iters"] == info2[r]["iters"]
    assert rel_l2(Pb.cpu().numpy(), Ps.cpu().numpy()) < 1e-13
    assert rel_l2(Pb.cpu().numpy(), exact) < 1e-8


def test_solve_batch_refined(sphere16_cldr):
    torch, dda = need_gpu()
    p, prob, prop, pol, exact = sphere16_cldr
    opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_CLDR, prec=dda.DDA_FP32_REFINED, tol=1e-8,
                maxiter=3000, inner_tol=1e-4)
    P = torch.zeros((len(prop), 3, p.n_occ), dtype=torch.complex128, device="cuda")
    st, info = dda.dda_solve_batch(p.h, opts, prop, pol, P)
    assert st == 0
    for r in range(len(prop)):
        assert info[r]["rel_res_true"] < 1e-8 and info[r]["outer"] >= 2
        assert info[r]["matvecs_fp64"] == info[r]["outer"]
    assert rel_l2(P.cpu().numpy(), exact) < 1e-6
    # other solvers are refused
    with pytest.raises(dda.DDAError) as ei:
        dda.dda_solve_batch(p.h, dict(opts, solver=dda.DDA_BICGSTAB), prop, pol, P)
    assert ei.value.status == dda.DDA_ERR_ARG


def test_solve_many_equals_one_by_one():
    """Particles in parallel host threads on their own streams give the same
    results as one dda_solve_batch call per particle."""
    torch, dda = need_gpu()
    parts = [(inputs.sphere(10), 1.3 + 0.01j), (inputs.ellipsoid(12, 8, 6), 1.5),
             (inputs.cube(6, 6, 6), 1.2 + 0.1j)]
    opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_CLDR, prec=dda.DDA_FP32_REFINED, tol=1e-6,
                maxiter=2000, inner_tol=1e-4)
    hs, props, pols, Ps, streams = [], [], [], [], []
    for k, (occ, m) in enumerate(parts):
        s = torch.cuda.Stream()
        p = dda.Particle(occ, [m], 0.45, stream=s)
        prop, pol = _orientations(2, 20 + k)
        hs.append(p); props.append(prop); pols.append(pol); streams.append(s)
        Ps.append(torch.zeros((len(prop), 3, p.n_occ), dtype=torch.complex128, device="cuda"))
    torch.cuda.synchronize()
    st, sts, infos = dda.dda_solve_many([p.h for p in hs], opts, props, pols, Ps, n_threads=2)
    assert st == 0 and sts == [0, 0, 0]
    for k, p in enumerate(hs):
        Q = torch.zeros_like(Ps[k])
        st1, info1 = dda.dda_solve_batch(p.h, opts, props[k], pols[k], Q)
        assert torch.equal(Q, Ps[k])
        assert [i["iters"] for i in info1] == [i["iters"] for i in infos[k]]
        assert all(i["rel_res_true"] < 1e-6 for i in infos[k])
        p.close()
    with pytest.raises(dda.DDAError):       # the same handle twice is refused
        q = dda.Particle(inputs.cube(4, 4, 4), [1.2], 0.4)
        with q:
            P = torch.zeros((2, 3, q.n_occ), dtype=torch.complex128, device="cuda")
            dda.dda_solve_many([q.h, q.h], opts, [props[0], props[0]], [pols[0], pols[0]], [P, P])



@pytest.mark.parametrize("prec_name", ["fp64", "fp32_refined"])
def test_graph_replayed_blocks_equal_launched_ones(prec_name):
    """On a stream of its own a handle's batched QMR-CS runs its blocks of 8
    steps as a replayed CUDA graph; on the legacy default stream (which cannot
    be captured) it launches them one by one.  Both give the same
    polarizations, bit for bit, and the same iteration counts."""
    torch, dda = need_gpu()
    occ = inputs.sphere(16)
    prop, pol = _orientations(2, 11)
    prec = dda.PREC[prec_name]
    opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_CLDR, prec=prec, tol=1e-9, maxiter=400,
                inner_tol=1e-3)
    out = []
    s = torch.cuda.Stream()
    for stream in (0, s):
        p = dda.Particle(occ, [1.6 + 0.05j], 0.5, stream=stream)
        with p:
            dda.dda_build_Dmatrix(p.h, prec)
            P = torch.zeros((len(prop), 3, p.n_occ), dtype=torch.complex128, device="cuda")
            torch.cuda.synchronize()
            st, info = dda.dda_solve_batch(p.h, opts, prop, pol, P)
            torch.cuda.synchronize()
            assert st == dda.DDA_OK, info
            out.append((P.cpu(), [i["iters"] for i in info]))
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
