"""Run a few interaction-matrix products on one sphere, for profilers.

    python -m paper_0704_0037_gb300.profile_case --n 134 --prec fp32 --products 3

Builds the sphere lattice (x = 40, m = 1.05 by default, LDR, incidence +z),
the D-matrix, and applies the product --products times to a seeded random
vector on cuda:0, then prints the mean time per product (CUDA events).
"""
import argparse
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=134)
    ap.add_argument("--x", type=float, default=40.0)
    ap.add_argument("--m", type=float, default=1.05)
    ap.add_argument("--prec", choices=["fp32", "fp64", "df"], default="fp32",
                    help="fp32: complex64 product; fp64: complex128; df: the double-float "
                         "product of the FP32-refined form (complex128 vectors)")
    ap.add_argument("--products", type=int, default=3)
    a = ap.parse_args(argv)
    import torch

    from paper_0704_0037_gb300 import build, dda, inputs
    build.build()
    torch.cuda.set_device(0)
    occ = inputs.sphere(a.n)
    with dda.Particle(occ, [a.m], a.x, volume_corrected=True) as p:
        prec = {"fp32": dda.DDA_FP32_REFINED, "fp64": dda.DDA_FP64, "df": dda.DDA_FP64_PAIR}[a.prec]
        dt = torch.complex64 if a.prec == "fp32" else torch.complex128
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP64 if a.prec == "fp64" else dda.DDA_FP32_REFINED)
        dda.dda_set_beta(p.h, dda.DDA_LDR, [(0, 0, 1)], [(1, 0, 0)])
        x = torch.from_numpy(inputs.random_vectors(1, 1, p.n_occ)).to("cuda", dt)
        y = torch.empty_like(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.products):
            dda.dda_matvec(p.h, prec, x, y)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / a.products
        print(f"n={a.n} grid={p.grid} n_occ={p.n_occ} prec={a.prec} ms_per_product={ms:.4f}")
        assert np.isfinite(y.abs().max().item())


if __name__ == "__main__":
    sys.exit(main())
