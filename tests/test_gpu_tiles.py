"""Tile variants of the register-resident product passes and their autotuner.

Every variant (lines per block of the y forward, fused z and y inverse passes)
computes each line with the same arithmetic, so the product must agree bit for
bit across variants, in every arithmetic and for the adjoint; the autotuner
(run by the D-matrix build) leaves a valid choice, and a pinned choice
survives a rebuild.
"""
import itertools

import pytest

from paper_0704_0037_gb300 import inputs

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

LATTICES = [("sphere16", inputs.sphere(16), [1.5], (32, 32, 32)),
            ("ellipsoid33x20x17", inputs.ellipsoid(33, 20, 17), [1.33 + 0.01j], (80, 40, 40)),
            ("ellipsoid40x36x12", inputs.ellipsoid(40, 36, 12), [1.2], (80, 80, 32))]
VARIANTS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]


@pytest.mark.parametrize("name,occ,m,grid", LATTICES, ids=[c[0] for c in LATTICES])
@pytest.mark.parametrize("form", ["fp32", "fp32_adjoint", "double_float", "fp64"])
def test_every_tile_variant_gives_the_same_product(name, occ, m, grid, form):
    torch, dda = need_gpu()
    p = dda.Particle(occ, m, 0.7)
    with p:
        assert p.grid == grid
        build = dda.DDA_FP64 if form == "fp64" else dda.DDA_FP32_REFINED
        dda.dda_build_Dmatrix(p.h, build)
        prec = {"fp32": dda.DDA_FP32_REFINED, "fp32_adjoint": dda.DDA_FP32_REFINED,
                "double_float": dda.DDA_FP64_PAIR, "fp64": dda.DDA_FP64}[form]
        # the autotuner chose a variant for each pass
        tuned = dda.dda_get_pass_tiles(p.h, prec)
        assert all(t in (0, 1) for t in tuned), tuned
        dda.dda_set_beta(p.h, dda.DDA_CLDR, [(0.0, 0.0, 1.0), (0.6, 0.0, 0.8)],
                         [(1.0, 0.0, 0.0), (0.8, 0.0, -0.6)])
        dt = torch.complex64 if prec == dda.DDA_FP32_REFINED else torch.complex128
        x = torch.from_numpy(inputs.random_vectors(3, 2, p.n_occ)).to("cuda", dt)
        f = dda.dda_matvec_adjoint if form == "fp32_adjoint" else dda.dda_matvec
        ys = []
        for v in VARIANTS:
            dda.dda_set_pass_tiles(p.h, prec, v)
            assert dda.dda_get_pass_tiles(p.h, prec) == v
            y = torch.empty_like(x)
            f(p.h, prec, x, y, 2)
            torch.cuda.synchronize()
            ys.append(y)
        for v, y in zip(VARIANTS[1:], ys[1:]):
            assert torch.equal(y, ys[0]), v


# the z pass of the long complex64 lines (512 = 16 x 32, 1080 = 30 x 36:
# fewer columns per block), the other axes Stockham
LONG_Z = [("ellipsoid6x5x256", inputs.ellipsoid(6, 5, 256), 512),
          ("ellipsoid4x3x540", inputs.ellipsoid(4, 3, 540), 1080)]


@pytest.mark.parametrize("name,occ,mz", LONG_Z, ids=[c[0] for c in LONG_Z])
@pytest.mark.parametrize("adjoint", [False, True], ids=["product", "adjoint"])
def test_long_z_tile_variants_give_the_same_product(name, occ, mz, adjoint):
    torch, dda = need_gpu()
    p = dda.Particle(occ, [1.4 + 0.02j], 0.6)
    with p:
        assert p.grid[2] == mz
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        assert dda.dda_get_pass_tiles(p.h, dda.DDA_FP32_REFINED)[1] in (0, 1)
        dda.dda_set_beta(p.h, dda.DDA_LDR, [(0.0, 0.0, 1.0)], [(1.0, 0.0, 0.0)])
        x = torch.from_numpy(inputs.random_vectors(4, 1, p.n_occ)).to("cuda", torch.complex64)
        f = dda.dda_matvec_adjoint if adjoint else dda.dda_matvec
        ys = []
        for v in ((0, 0, 0), (0, 1, 0)):
            dda.dda_set_pass_tiles(p.h, dda.DDA_FP32_REFINED, v)
            y = torch.empty_like(x)
            f(p.h, dda.DDA_FP32_REFINED, x, y, 1)
            torch.cuda.synchronize()
            ys.append(y)
        assert torch.equal(ys[0], ys[1])


def test_pinned_tiles_survive_a_rebuild_and_bad_values_are_refused():
    torch, dda = need_gpu()
    p = dda.Particle(inputs.sphere(16), [1.5], 0.7)
    with p:
        assert dda.dda_get_pass_tiles(p.h, dda.DDA_FP32_REFINED) == (-1, -1, -1)
        dda.dda_set_pass_tiles(p.h, dda.DDA_FP32_REFINED, (1, 0, -1))
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        t = dda.dda_get_pass_tiles(p.h, dda.DDA_FP32_REFINED)
        assert t[:2] == (1, 0) and t[2] in (0, 1)
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        assert dda.dda_get_pass_tiles(p.h, dda.DDA_FP32_REFINED)[:2] == (1, 0)
        for bad in ((2, 0, 0), (0, -2, 0)):
            with pytest.raises(dda.DDAError) as ei:
                dda.dda_set_pass_tiles(p.h, dda.DDA_FP32_REFINED, bad)
            assert ei.value.status == dda.DDA_ERR_ARG
        with pytest.raises(dda.DDAError) as ei:
            dda.dda_set_pass_tiles(p.h, 7, (0, 0, 0))
        assert ei.value.status == dda.DDA_ERR_ARG
        # back to the autotuner
        dda.dda_set_pass_tiles(p.h, dda.DDA_FP32_REFINED, None)
        assert dda.dda_get_pass_tiles(p.h, dda.DDA_FP32_REFINED) == (-1, -1, -1)
