"""Training of the learned right preconditioner (dda_pcnet_* in the C-ABI).

Host-side orchestration only: every product, solve, network pass and Adam
step runs in libdda.so.  Pairs come from the solver's own runs (north-star
pattern; the paper trains nothing): for each training particle, the
FP32-refined QMR-CS solution x* to a tight tolerance, and early QMR-CS
iterates x_k (k products), give e = x* - x_k and r = A e (dda_pcnet_pair);
the network learns r -> e.
"""
import time

import numpy as np

from . import dda, inputs


def train(net, count=128, n=64, ks=(8, 32, 96), tol_star=1e-6, lr=1e-3, epochs=2, seed=704037,
          log=None):
    """Train `net` on `count` particles; returns a summary dict."""
    import torch
    prop, pol = [(0.0, 0.0, 1.0)], [(1.0, 0.0, 0.0)]
    losses, t0, pairs_done, mv = [], time.perf_counter(), 0, 0
    for i, (occ, m, kd) in enumerate(inputs.training_particles(count, n, seed)):
        with dda.Particle(occ, [m], kd) as p:
            dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
            Ps = torch.zeros((1, 3, p.n_occ), dtype=torch.complex128, device="cuda")
            st, info, _ = dda.dda_solve(p.h, dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_LDR,
                                                  prec=dda.DDA_FP32_REFINED, tol=tol_star,
                                                  maxiter=20000, inner_tol=1e-3), prop, pol, Ps)
            mv += info[0]["matvecs"]
            pairs = []
            for k in ks:
                Pk = torch.zeros_like(Ps)
                _, ik, _ = dda.dda_solve(p.h, dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_LDR,
                                                   prec=dda.DDA_FP64, tol=1e-12, maxiter=k), prop, pol, Pk)
                mv += ik[0]["matvecs"]
                r = torch.empty((3, p.n_occ), dtype=torch.complex128, device="cuda")
                e = torch.empty_like(r)
                dda.dda_pcnet_pair(p.h, dda.DDA_LDR, prop, pol, Ps[0], Pk[0], r, e)
                pairs.append((r, e))
            z = torch.empty((3, p.n_occ), dtype=torch.complex128, device="cuda")
            for _ in range(epochs):
                for r, e in pairs:
                    losses.append(net.train_step(p.h, r, e, z, lr))
                    pairs_done += 1
        if log and (i + 1) % 16 == 0:
            log(f"particle {i + 1}/{count}: mean loss of the last 48 steps "
                f"{np.mean(losses[-48:]):.4f}")
    return {"particles": count, "box": n, "pairs_per_particle": len(ks), "epochs": epochs,
            "train_steps": pairs_done, "solver_products": mv, "seconds": time.perf_counter() - t0,
            "loss_first16": float(np.mean(losses[:16])), "loss_last16": float(np.mean(losses[-16:]))}
