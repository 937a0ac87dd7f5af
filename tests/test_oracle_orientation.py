"""Pins for the oracle's orientation averaging (Sec. 2, orientation averaging
over Euler angles): rotation conventions checked against rotated lattices,
a closed form for one dipole, and the rotation invariance of the average."""
import math

import numpy as np
import pytest

from oracle import dda, lattice, observables, orientation, polarizability, system


def _dense_solve(prob):
    return lambda beta, b: system.solve_dense(prob.pos, beta, prob.kd, b)


def _rotate_y90(occ):
    """Occupancy of the lattice turned by +90 degrees about y: (x, y, z) -> (z, y, -x)."""
    return np.ascontiguousarray(np.flip(occ.transpose(2, 1, 0), axis=0))


def _rotate_z90(occ):
    """(x, y, z) -> (-y, x, z)."""
    return np.ascontiguousarray(np.flip(occ.transpose(0, 2, 1), axis=2))


@pytest.mark.parametrize("rot", ["y", "z", "zy"])
def test_oriented_scattering_equals_rotated_lattice(rot):
    """Orientation R applied to the particle gives the same Q and Mueller
    matrix as the laboratory lattice R(particle) at orientation I."""
    rng = np.random.default_rng(3)
    occ = (rng.random((3, 4, 5)) < 0.7).astype(np.uint8) * (1 + (rng.random((3, 4, 5)) < 0.4))
    occ[1, 1, 1] = 1
    m = [1.5 + 0.1j, 1.2]
    kd = 0.6
    if rot == "y":
        R, occ_lab = orientation.rot_y(math.pi / 2), _rotate_y90(occ)
    elif rot == "z":
        R, occ_lab = orientation.rot_z(math.pi / 2), _rotate_z90(occ)
    else:
        R, occ_lab = orientation.rot_z(math.pi / 2) @ orientation.rot_y(math.pi / 2), \
            _rotate_z90(_rotate_y90(occ))
    pp = dda.Problem(occ, m, kd)
    pl = dda.Problem(occ_lab, m, kd)
    # the laboratory lattice is the rotated particle lattice, materials included
    a = sorted(map(tuple, np.round(np.c_[pp.pos @ R.T, pp.mat], 9)))
    b = sorted(map(tuple, np.round(np.c_[pl.pos, pl.mat], 9)))
    assert a == b
    th = np.arange(0.0, 181.0, 20.0)
    for presc in ("cldr", "rr"):
        qe1, qa1, M1 = orientation.oriented(pp, 1.0, presc, R, th, 3, _dense_solve(pp))
        qe2, qa2, M2 = orientation.oriented(pl, 1.0, presc, np.eye(3), th, 3, _dense_solve(pl))
        assert abs(qe1 - qe2) < 1e-12 * abs(qe2) and abs(qa1 - qa2) < 1e-12 * abs(qe2)
        assert np.abs(M1 - M2).max() < 1e-12 * np.abs(M2).max()


def test_single_dipole_average_closed_form():
    """One isotropic dipole: every orientation scatters alike; with
    P = alpha e, S2 = -i kd^3 alpha cos(t), S1 = -i kd^3 alpha, S3 = S4 = 0, so
    M11 = k6 (1 + cos^2 t)/2, M12 = -k6 sin^2 t / 2, M33 = M44 = k6 cos t,
    k6 = kd^6 |alpha|^2."""
    occ = np.ones((1, 1, 1), dtype=np.uint8)
    kd = 0.4
    prob = dda.Problem(occ, [1.5 + 0.2j], kd)
    th = np.arange(0.0, 181.0, 15.0)
    qe, qa, M = orientation.average(prob, 1.0, "rr", 4, 3, 5, th, _dense_solve(prob))
    alpha = polarizability.alpha_diag(1.5 + 0.2j, kd, "rr")[0]
    k6 = kd ** 6 * abs(alpha) ** 2
    t = np.deg2rad(th)
    ref = np.zeros((th.size, 4, 4))
    ref[:, 0, 0] = ref[:, 1, 1] = 0.5 * k6 * (1 + np.cos(t) ** 2)
    ref[:, 0, 1] = ref[:, 1, 0] = -0.5 * k6 * np.sin(t) ** 2
    ref[:, 2, 2] = ref[:, 3, 3] = k6 * np.cos(t)
    assert np.abs(M - ref).max() < 1e-13 * k6
    assert abs(qe - 4 * kd ** 3 * alpha.imag) < 1e-14


def test_average_is_rotation_invariant():
    """A small dimer along x and the same dimer along z: the averages over
    all orientations agree; the fixed quadrature converges geometrically
    (1e-8 at 8 x 10 x 8 nodes, 1e-14 at 16 x 20 x 12)."""
    kd = 0.25
    th = np.arange(0.0, 181.0, 30.0)
    out = []
    for occ in (np.ones((1, 1, 2), dtype=np.uint8), np.ones((2, 1, 1), dtype=np.uint8)):
        prob = dda.Problem(occ, [2.0 + 0.5j], kd)
        out.append(orientation.average(prob, 1.0, "rr", 12, 16, 20, th, _dense_solve(prob)))
    (qe1, qa1, M1), (qe2, qa2, M2) = out
    assert abs(qe1 - qe2) < 1e-12 * qe1
    assert np.abs(M1 - M2).max() < 1e-12 * np.abs(M1).max()


def test_ldr_is_refused():
    prob = dda.Problem(np.ones((1, 1, 2), dtype=np.uint8), [1.5], 0.3)
    with pytest.raises(ValueError):
        orientation.oriented(prob, 1.0, "ldr", np.eye(3), [0.0], 1, _dense_solve(prob))
