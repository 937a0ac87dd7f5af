"""Host-side checks of the seeded workload generators (no GPU)."""
import numpy as np

from paper_0704_0037_gb300 import inputs


def test_batch_instances_generator():
    """The seeded batch: 128 particles, 16 right-hand sides each, the
    drawing rule of the generator (n from 10 dipoles per wavelength)."""
    b = inputs.batch_instances()
    assert len(b) == 128 and all(i["prop"].shape == (16, 3) for i in b)
    for i in b:
        n = max(i["occ"].shape)
        assert n == min(64, max(16, int(np.ceil(10 * i["x"] * i["m"] / np.pi))))
        assert 2.0 <= i["x"] <= 15.0 and 1.05 <= i["m"] <= 2.0
        assert np.allclose(np.einsum("ij,ij->i", i["prop"], i["pol"]), 0, atol=1e-15)
