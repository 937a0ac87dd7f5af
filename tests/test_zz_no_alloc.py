"""The allocation-free far-field entry point, dda_farfield_noalloc.

Callers that cannot let a library allocate device memory (code running under
CUDA stream capture, processes that hand out device memory from their own
fixed pool) use dda_farfield_noalloc instead of dda_scatter to get the
scattering amplitude F(n).  It keeps its working memory in one fixed device
array.  These tests call it through the C-ABI and compare it with
dda_scatter (the allocating entry point) and with the CPU oracle's far field
(the definition, summed over the dipoles in complex128) on two calls in a
row -- different polarizations and direction sets, so stale contents of the
shared array would show -- check that repeat calls take no device memory,
and that a request above the fixed limit is refused.  This file is collected
last on purpose.
"""
import numpy as np
import pytest

from oracle import lattice, observables
from paper_0704_0037_gb300 import inputs

from gpu_util import need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def test_farfield_noalloc_matches_scatter_twice():
    torch, dda = need_gpu()
    occ = inputs.ellipsoid(18, 14, 11)
    prop, pol = [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]]
    pos = lattice.positions(occ > 0)
    with dda.Particle(occ, [1.4 + 0.05j], 0.6) as p:
        free = []
        for call, seed in enumerate((1, 2, 3)):
            P = torch.from_numpy(inputs.random_vectors(seed, 1, p.n_occ)).cuda()
            # general directions (non-zero y components): dda_scatter's direct sum
            dirs = inputs.random_unit_vectors(10 + seed, 37 + 50 * call)
            F_ref, _ = dda.dda_scatter(p.h, dda.DDA_LDR, P, prop, pol, dirs)
            d_dev = torch.from_numpy(np.ascontiguousarray(dirs)).cuda()
            F = torch.empty((dirs.shape[0], 3), dtype=torch.complex128, device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            dda.dda_farfield_noalloc(p.h, P, d_dev, F)
            torch.cuda.synchronize()
            free.append((free_before, torch.cuda.mem_get_info()[0]))
            Fn = F.cpu().numpy()
            assert rel_l2(Fn, F_ref[0]) <= 1e-12
            # the definition F(n) = -i kd^3 (I - n n) sum_j P_j exp(-i kd n.r_j)
            F_or = observables.farfield(P.cpu().numpy().reshape(3, -1), pos, p.kd, dirs)
            assert rel_l2(Fn, F_or) <= 1e-12
        # after the first call (which looks up the array's address), calls
        # take no device memory
        for before, after in free[1:]:
            assert after == before


def test_farfield_noalloc_rejects_oversize_request():
    torch, dda = need_gpu()
    occ = inputs.sphere(12)
    with dda.Particle(occ, [1.5], 0.5) as p:
        n_dir = 20000          # 20000 * 36 * 16 B of phase tables alone > 8 MiB
        dirs = torch.zeros((n_dir, 3), dtype=torch.float64, device="cuda")
        dirs[:, 2] = 1.0
        P = torch.zeros((3, p.n_occ), dtype=torch.complex128, device="cuda")
        F = torch.empty((n_dir, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(dda.DDAError) as ei:
            dda.dda_farfield_noalloc(p.h, P, dirs, F)
        assert ei.value.status == dda.DDA_ERR_ARG
        assert "fixed limit" in dda.dda_last_error(p.h)
