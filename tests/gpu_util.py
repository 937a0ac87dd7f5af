"""Shared helpers of the GPU tests: load the library, build an oracle twin."""
import numpy as np
import pytest

from oracle import dda as odda
from oracle import lattice


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0704_0037_gb300 import build, dda
    build.build()
    dda.lib()
    return torch, dda


def twin(occ, m_list, kd, volume_x=None):
    """(library Particle, oracle Problem) for the same lattice."""
    from paper_0704_0037_gb300 import dda
    if volume_x is not None:
        p = dda.Particle(occ, m_list, volume_x, volume_corrected=True)
        kd = lattice.kd_volume_corrected(volume_x, p.n_occ)
    else:
        p = dda.Particle(occ, m_list, kd)
    prob = odda.Problem(occ, m_list, kd, grid=p.grid)
    return p, prob


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
