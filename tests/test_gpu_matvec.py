"""GPU parity of the FFT interaction-matrix product (Eq. 2-3) against the oracle.

Tolerances: relative L2 <= 1e-12 for complex128, <= 1e-5 for complex64
(the accuracy the two forms are built for); at full size the comparison is on sampled outputs that
the oracle computes one by one by the direct sum.
"""
import numpy as np
import pytest

from paper_0704_0037_gb300 import inputs

from gpu_util import direct_sum_rows, need_gpu, rel_l2, sample_dipoles, twin

pytestmark = pytest.mark.gpu

def _gaps():
    """A lattice whose occupied rows leave gaps: empty z planes, planes whose
    span of occupied rows holds empty rows, planes of one dipole, and more
    planes than one block of rows covers (16 x 20 x 18 box, grid 32 x 40 x 40)."""
    occ = np.zeros((18, 20, 16), np.uint8)       # (z, y, x)
    occ[2:6, 1:4, 3:9] = 1
    occ[3, 12, :] = 2                            # plane 3: rows 1-3 and 12
    occ[9, 10, 7] = 1                            # plane 9: one dipole
    occ[12:16, 15:20, 5:12] = 2
    occ[14, 0, 15] = 1                           # plane 14: rows 0 and 15-19
    return occ


CASES = [
    ("sphere1", inputs.sphere(1), [1.5]),
    ("sphere2", inputs.sphere(2), [1.5]),
    ("sphere3", inputs.sphere(3), [1.5]),
    ("sphere5", inputs.sphere(5), [1.3 + 0.1j]),
    ("layered7", inputs.layered_sphere(7, 3), [1.5, 1.2 + 0.05j, 2.0]),
    ("cube3x5x7", inputs.cube(3, 5, 7), [1.4]),
    ("ellipsoid12x9x6", inputs.ellipsoid(12, 9, 6), [1.6]),
    ("random6x5x4", inputs.random_occupancy(6, 5, 4, 0.6, seed=11, n_mat=2), [1.5, 1.1 + 0.2j]),
    ("sphere16", inputs.sphere(16), [1.5]),
    ("ellipsoid33x20x17", inputs.ellipsoid(33, 20, 17), [1.33]),
    ("random40x9x23", inputs.random_occupancy(40, 9, 23, 0.3, seed=3, n_mat=3), [1.5, 1.05, 2.0 + 0.1j]),
    ("gaps16x20x18", _gaps(), [1.5, 1.2 + 0.05j]),
]


def _run(p, prob, prec, presc, props, pols, x, adjoint=False):
    torch, dda = need_gpu()
    dda.dda_set_beta(p.h, dda.POL[presc], props, pols)
    dt = torch.complex64 if prec == dda.DDA_FP32_REFINED else torch.complex128
    xd = torch.from_numpy(x).to(device="cuda", dtype=dt)
    yd = torch.empty_like(xd)
    f = dda.dda_matvec_adjoint if adjoint else dda.dda_matvec
    f(p.h, prec, xd, yd, x.shape[0])
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = []
    for r in range(x.shape[0]):
        beta = prob.beta(presc, props[r], pols[r])
        from oracle.fft_matvec import matvec_fft
        ref.append(matvec_fft(prob.occ, beta, prob.dmat(), x[r], conj=adjoint))
    return y, np.stack(ref)


@pytest.mark.parametrize("name,occ,m", CASES, ids=[c[0] for c in CASES])
def test_matvec_fp64(name, occ, m):
    torch, dda = need_gpu()
    p, prob = twin(occ, m, 0.55)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP64)
        x = inputs.random_vectors(7, 1, p.n_occ)
        y, ref = _run(p, prob, dda.DDA_FP64, "cldr", [(0.6, 0.0, 0.8)], [(0.8, 0.0, -0.6)], x)
        assert rel_l2(y, ref) <= 1e-12


@pytest.mark.parametrize("name,occ,m", CASES, ids=[c[0] for c in CASES])
def test_matvec_fp32(name, occ, m):
    torch, dda = need_gpu()
    p, prob = twin(occ, m, 0.55)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        x = inputs.random_vectors(8, 1, p.n_occ)
        y, ref = _run(p, prob, dda.DDA_FP32_REFINED, "ldr", [(0, 0, 1)], [(1, 0, 0)], x)
        assert rel_l2(y, ref) <= 1e-5


DF_CASES = [
    ("sphere16", inputs.sphere(16), [1.5]),                                      # 32^3
    ("random16x64x16", inputs.random_occupancy(16, 64, 16, 0.5, seed=4, n_mat=2),
     [1.5 + 0.1j, 2.0]),                                                        # 32 x 128 x 32
    ("ellipsoid64x16x16", inputs.ellipsoid(64, 16, 16), [1.33]),                 # 128 x 32 x 32
    ("gaps16x20x18", _gaps(), [1.5, 1.2 + 0.05j]),                              # 32 x 40 x 40
]


@pytest.mark.parametrize("name,occ,m", DF_CASES, ids=[c[0] for c in DF_CASES])
def test_matvec_double_float(name, occ, m):
    """The double-float product (FP32_REFINED build on a grid with
    register-resident passes; used for the refinement residuals) is within
    FP64 tolerance of the oracle, for several right-hand sides at once."""
    torch, dda = need_gpu()
    p, prob = twin(occ, m, 0.55)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        x = inputs.random_vectors(9, 2, p.n_occ)
        props = [(0.6, 0.0, 0.8), (0.0, 0.0, 1.0)]
        pols = [(0.8, 0.0, -0.6), (0.0, 1.0, 0.0)]
        y, ref = _run(p, prob, dda.DDA_FP64_PAIR, "cldr", props, pols, x)
        assert rel_l2(y, ref) <= 1e-12
        # the FP64 octant derived from the double-float build serves FP64 products
        y64, _ = _run(p, prob, dda.DDA_FP64, "cldr", props, pols, x)
        assert rel_l2(y64, ref) <= 1e-12


def test_double_float_needs_its_build():
    torch, dda = need_gpu()
    p, prob = twin(inputs.sphere(16), [1.5], 0.5)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP64)
        dda.dda_set_beta(p.h, dda.DDA_LDR, [(0, 0, 1)], [(1, 0, 0)])
        x = torch.zeros((1, 3, p.n_occ), dtype=torch.complex128, device="cuda")
        with pytest.raises(dda.DDAError) as ei:
            dda.dda_matvec(p.h, dda.DDA_FP64_PAIR, x, torch.empty_like(x))
        assert ei.value.status == dda.DDA_ERR_STATE


def test_matvec_multi_rhs_and_adjoint():
    torch, dda = need_gpu()
    occ = inputs.ellipsoid(14, 11, 9)
    p, prob = twin(occ, [1.7 + 0.3j], 0.45)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP64)
        props = inputs.random_unit_vectors(4, 3)
        pols = np.stack([inputs.perpendicular_pols(a)[0] for a in props])
        x = inputs.random_vectors(9, 3, p.n_occ)
        y, ref = _run(p, prob, dda.DDA_FP64, "cldr", props, pols, x)
        assert rel_l2(y, ref) <= 1e-12
        y, ref = _run(p, prob, dda.DDA_FP64, "cldr", props, pols, x, adjoint=True)
        assert rel_l2(y, ref) <= 1e-12


# Padded lengths under the default engine (compiled lengths within 1.35 times
# the smallest 7-smooth one; the Stockham engine keeps the 7-smooth ones):
ENGINE_CASES = [
    ("sphere16_M32", inputs.sphere(16)),
    ("sphere32_M64", inputs.sphere(32)),
    ("sphere64_M128", inputs.sphere(64)),
    ("ellipsoid64x60x33", inputs.ellipsoid(64, 60, 33)),   # 128, 128, 80
    ("ellipsoid70x128x100", inputs.ellipsoid(70, 128, 100)),  # 140 (Stockham), 256, 256
    ("ellipsoid20x24x128", inputs.ellipsoid(20, 24, 128)),    # 40, 48, 256
    ("ellipsoid134x12x134", inputs.ellipsoid(134, 12, 134)),  # 270, 32, 270
    ("ellipsoid37x23x45", inputs.ellipsoid(37, 23, 45)),      # 80, 48, 96: the added lengths
    # complex64 register-resident passes of the large grids (512 and 1080) on
    # each axis, the other axes Stockham
    ("ellipsoid256x6x5", inputs.ellipsoid(256, 6, 5)),
    ("ellipsoid5x256x6", inputs.ellipsoid(5, 256, 6)),
    ("ellipsoid6x5x256", inputs.ellipsoid(6, 5, 256)),
    ("ellipsoid540x4x3", inputs.ellipsoid(540, 4, 3)),
    ("ellipsoid3x540x4", inputs.ellipsoid(3, 540, 4)),
    ("ellipsoid4x3x540", inputs.ellipsoid(4, 3, 540)),
    # z fast (256) under rows of an odd padded x length (7): element-wise staging
    ("ellipsoid4x3x128", inputs.ellipsoid(4, 3, 128)),
]


@pytest.mark.parametrize("name,occ", ENGINE_CASES, ids=[c[0] for c in ENGINE_CASES])
@pytest.mark.parametrize("prec_name", ["fp64", "fp32_refined"])
def test_register_engine_matches_stockham_and_oracle(name, occ, prec_name):
    """The register-resident passes (compiled lengths 32, 64, 128, 256, 270;
    complex64 also 512 and 1080) and the shared-memory Stockham passes give
    the same product, and both match
    the oracle."""
    torch, dda = need_gpu()
    prec = dda.PREC[prec_name]
    dt = torch.complex128 if prec == dda.DDA_FP64 else torch.complex64
    tol = 1e-12 if prec == dda.DDA_FP64 else 1e-5
    ys = {}
    for engine in ("auto", "stockham"):
        p, prob = twin(occ, [1.3 + 0.02j], 0.5)
        with p:
            dda.dda_set_fft_engine(p.h, dda.DDA_ENGINE_STOCKHAM if engine == "stockham"
                                   else dda.DDA_ENGINE_AUTO)
            dda.dda_build_Dmatrix(p.h, prec)
            dda.dda_set_beta(p.h, dda.DDA_CLDR, [(0.6, 0.0, 0.8)], [(0.8, 0.0, -0.6)])
            x = inputs.random_vectors(13, 1, p.n_occ)
            xd = torch.from_numpy(x).to("cuda", dt)
            yd = torch.empty_like(xd)
            dda.dda_matvec(p.h, prec, xd, yd)
            yd2 = torch.empty_like(xd)
            dda.dda_matvec_adjoint(p.h, prec, xd, yd2)
            ys[engine] = (yd.cpu().numpy()[0], yd2.cpu().numpy()[0])
    from oracle.fft_matvec import matvec_fft
    beta = prob.beta("cldr", (0.6, 0.0, 0.8), (0.8, 0.0, -0.6))
    ref = matvec_fft(prob.occ, beta, prob.dmat(), x[0])
    ref_h = matvec_fft(prob.occ, beta, prob.dmat(), x[0], conj=True)
    for engine, (y, yh) in ys.items():
        assert rel_l2(y, ref) <= tol, engine
        assert rel_l2(yh, ref_h) <= tol, engine
    assert rel_l2(ys["auto"][0], ys["stockham"][0]) <= tol


def test_matvec_is_deterministic():
    torch, dda = need_gpu()
    occ = inputs.sphere(20)
    p, prob = twin(occ, [1.5], 0.5)
    with p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        dda.dda_set_beta(p.h, dda.DDA_LDR, [(0, 0, 1)], [(1, 0, 0)])
        for prec, dt in ((dda.DDA_FP64, torch.complex128), (dda.DDA_FP32_REFINED, torch.complex64)):
            xd = torch.from_numpy(inputs.random_vectors(2, 1, p.n_occ)).to("cuda", dt)
            y1, y2 = torch.empty_like(xd), torch.empty_like(xd)
            dda.dda_matvec(p.h, prec, xd, y1)
            dda.dda_matvec(p.h, prec, xd, y2)
            assert torch.equal(y1, y2)


@pytest.mark.slow
@pytest.mark.parametrize("prec_name", ["fp64", "fp32_refined", "fp64_pair"])
def test_matvec_full_size_sampled(prec_name):
    """Sphere x = 40, m = 1.05 at 134^3 (1,260,552 dipoles), padded 270^3:
    sampled outputs against the direct sum."""
    torch, dda = need_gpu()
    occ = inputs.sphere(134)
    p = dda.Particle(occ, [1.05], 40.0, volume_corrected=True)
    with p:
        assert p.n_occ == 1260552 and p.grid == (270, 270, 270)
        prec = dda.PREC[prec_name] if prec_name != "fp64_pair" else dda.DDA_FP64_PAIR
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP64 if prec == dda.DDA_FP64 else dda.DDA_FP32_REFINED)
        dda.dda_set_beta(p.h, dda.DDA_LDR, [(0, 0, 1)], [(1, 0, 0)])
        x = inputs.random_vectors(21, 1, p.n_occ)
        dt = torch.complex64 if prec == dda.DDA_FP32_REFINED else torch.complex128
        xd = torch.from_numpy(x).to("cuda", dt)
        yd = torch.empty_like(xd)
        dda.dda_matvec(p.h, prec, xd, yd)
        y = yd.cpu().numpy()[0]
        from oracle import dda as odda
        prob = odda.Problem(occ, [1.05], p.kd)
        beta = prob.beta("ldr", (0, 0, 1), (1, 0, 0))
        idx = sample_dipoles(occ, 32, 5)
        assert len(idx) == 32
        ref = direct_sum_rows(prob.pos, beta, prob.kd, x[0], idx)
        scale = np.sqrt(np.mean(np.abs(ref) ** 2))
        err = np.abs(y[:, idx] - ref).max() / scale
        assert err <= (1e-5 if prec == dda.DDA_FP32_REFINED else 1e-12), err
