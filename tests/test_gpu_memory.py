"""Device memory of the library: buffers a handle frees go to a per-process
cache and serve the next handle of the same size.  Reuse must not change any
result on any stream, and the cache must be releasable."""
import numpy as np
import pytest

from paper_0704_0037_gb300 import inputs

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _products(torch, dda, occ, stream=None):
    p = dda.Particle(occ, [1.5 + 0.02j], 3.0, volume_corrected=True, stream=stream)
    try:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        dda.dda_set_beta(p.h, dda.DDA_LDR, [(0, 0, 1)], [(1, 0, 0)])
        out = []
        for prec, dt in ((dda.DDA_FP64, torch.complex128), (dda.DDA_FP32_REFINED, torch.complex64),
                         (dda.DDA_FP64_PAIR, torch.complex128)):
            x = torch.from_numpy(inputs.random_vectors(3, 1, p.n_occ)).to("cuda", dt)
            y = torch.empty_like(x)
            dda.dda_matvec(p.h, prec, x, y)
            out.append(y)
        torch.cuda.synchronize()
        return [y.cpu().numpy() for y in out]
    finally:
        p.close()


def test_reused_buffers_give_identical_results():
    torch, dda = need_gpu()
    occ = inputs.sphere(16)
    first = _products(torch, dda, occ)
    for k in range(3):
        again = _products(torch, dda, occ)
        for a, b in zip(first, again):
            assert np.array_equal(a, b)
        if k == 1:
            assert dda.dda_release_cached_memory() == 0


def test_reuse_across_streams():
    """Handles on two different streams take over each other's cached blocks
    (each block waits on an event of the stream that freed it); every result
    matches the first, freshly allocated one bit for bit."""
    torch, dda = need_gpu()
    occ = inputs.sphere(16)
    ref = _products(torch, dda, occ)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(2):
        a = _products(torch, dda, occ, stream=s1)
        b = _products(torch, dda, occ, stream=s2)
        for r, u, v in zip(ref, a, b):
            assert np.array_equal(r, u)
            assert np.array_equal(r, v)


def test_solve_after_release_matches():
    torch, dda = need_gpu()
    occ = inputs.sphere(16)
    opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_LDR, prec=dda.DDA_FP32_REFINED, tol=1e-8,
                maxiter=500, inner_tol=1e-6)
    res = []
    for k in range(2):
        with dda.Particle(occ, [1.5], 3.0, volume_corrected=True) as p:
            dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
            P = torch.zeros((1, 3, p.n_occ), dtype=torch.complex128, device="cuda")
            st, info, _ = dda.dda_solve(p.h, opts, np.array([[0.0, 0.0, 1.0]]),
                                        np.array([[1.0, 0.0, 0.0]]), P)
            assert st == 0
            res.append(P.cpu().numpy())
        dda.dda_release_cached_memory()
    assert np.array_equal(res[0], res[1])
