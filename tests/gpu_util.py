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


def sample_dipoles(occ, count, seed):
    """`count` distinct dipole indices (x-fastest scan order) spread over the
    lattice for sampled parity: the first, middle and last dipole, both ends
    of randomly chosen rows (dipoles on the particle's surface, where the
    interaction sums are least symmetric), and random dipoles."""
    occ = np.asarray(occ) > 0
    nz, ny, nx = occ.shape
    per_row = occ.reshape(nz * ny, nx).sum(axis=1)
    off = np.concatenate([[0], np.cumsum(per_row)])
    n = int(off[-1])
    rng = np.random.default_rng(seed)
    picks = {0, n // 2, n - 1}
    rows = rng.permutation(np.nonzero(per_row)[0])
    for r in rows[: max(1, count // 3)]:
        picks.add(int(off[r]))
        picks.add(int(off[r + 1] - 1))
    while len(picks) < min(count, n):
        picks.add(int(rng.integers(0, n)))
    return np.array(sorted(picks)[:count] if len(picks) > count else sorted(picks))


def direct_sum_rows(pos, beta, kd, x, idx):
    """The oracle's direct sum (oracle.system.matvec_rows) at the sampled
    dipoles idx, one row per host thread (numpy releases the GIL in its array
    operations; threads, unlike forked processes, are safe next to CUDA)."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    from oracle import system
    workers = max(1, min(len(idx), os.cpu_count() or 1, 16))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        cols = list(ex.map(lambda i: system.matvec_rows(pos, beta, kd, x, [int(i)])[:, 0], idx))
    return np.stack(cols, axis=1)
