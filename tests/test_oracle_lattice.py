"""Pins for the oracle's lattice, occupancy and volume correction (O1/O2)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import lattice
from paper_0704_0037_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _float_sphere(n):
    # independent formulation: centre distance <= radius, in floating point
    c = np.arange(n) + 0.5 - n / 2.0
    d2 = c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2
    return d2 <= (n / 2.0) ** 2


@pytest.mark.parametrize("n,count", [(1, 1), (2, 8), (3, 19), (16, 2176), (64, 137376),
                                     (128, 1099136), (134, 1260552)])
def test_sphere_counts(n, count):
    occ = lattice.sphere_occupancy(n)
    assert int(occ.sum()) == count
    if n <= 64:
        assert np.array_equal(occ, _float_sphere(n))


@pytest.mark.parametrize("n", list(range(1, 70)))
def test_sphere_has_no_ties(n):
    # sum (2i+1-n)^2 never equals n^2, so the occupancy is unambiguous
    q = (2 * np.arange(n) + 1 - n) ** 2
    s = q[:, None, None] + q[None, :, None] + q[None, None, :]
    assert not np.any(s == n * n)


def test_sphere_fraction_tends_to_pi_over_6():
    for n, tol in [(32, 0.02), (134, 0.005)]:
        f = lattice.sphere_occupancy(n).mean()
        assert abs(f - math.pi / 6) < tol


def test_ellipsoid_reduces_to_sphere_and_cube():
    for n in (5, 8, 13):
        assert np.array_equal(lattice.ellipsoid_occupancy(n, n, n), lattice.sphere_occupancy(n))
    assert lattice.cube_occupancy(3, 5, 7).sum() == 105
    assert lattice.cube_occupancy(3, 5, 7).shape == (7, 5, 3)


def test_ellipsoid_axes():
    occ = lattice.ellipsoid_occupancy(9, 5, 3)
    iz, iy, ix = np.nonzero(occ)
    assert ix.min() == 0 and ix.max() == 8       # spans the long axis
    assert iz.min() >= 0 and iz.max() <= 2


def test_inputs_shapes_match_oracle():
    for n in (1, 2, 7, 16, 33):
        assert np.array_equal(inputs.sphere(n) > 0, lattice.sphere_occupancy(n))
    assert np.array_equal(inputs.ellipsoid(9, 6, 4) > 0, lattice.ellipsoid_occupancy(9, 6, 4))


def test_positions_order_and_centre():
    occ = lattice.cube_occupancy(3, 2, 2)
    pos = lattice.positions(occ)
    # x fastest, origin at the box centre, unit spacing
    assert np.allclose(pos[:4], [[-1, -0.5, -0.5], [0, -0.5, -0.5], [1, -0.5, -0.5], [-1, 0.5, -0.5]])
    sp = lattice.positions(lattice.sphere_occupancy(12))
    assert np.allclose(sp.sum(axis=0), 0.0)


def test_volume_correction():
    n_occ = 2176
    kd = lattice.kd_volume_corrected(3.0, n_occ)
    # N d^3 = (4/3) pi a^3  with  x = k a
    a_over_d = (3.0 * n_occ / (4.0 * math.pi)) ** (1.0 / 3.0)
    assert abs(kd * a_over_d - 3.0) < 1e-14
    assert abs(kd - 0.37319) < 5e-5


def test_size_rule_against_table1():
    """Sec. 3.1 / Table 1: the box count is about (3.18 x m)^3 at 10 dipoles per
    wavelength; with the printed lambda/(m d) the rule reproduces every row."""
    with open(os.path.join(GOLDEN, "table1.json")) as f:
        rows = json.load(f)["rows"]
    assert len(rows) == 24
    for r in rows:
        n = 3.18 * r["x"] * r["m"] * r["lambda_md"] / 10.0
        assert abs(n ** 3 / r["box_dipoles"] - 1.0) < 0.06, r
    # config sizes follow the rule
    assert inputs.size_rule_n(40.0, 1.05) == 134
