"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
include/dda.h declares, and its host-only logic is right.  No GPU work."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import observables
from paper_0704_0037_gb300 import build, dda, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return dda.lib()


def _declared():
    with open(os.path.join(ROOT, "include", "dda.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dda_[a-z_0-9A-Z]+)\s*\(", src)))


def test_header_and_binding_agree(L):
    declared = _declared()
    assert declared == sorted(dda.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def test_exports_are_c_symbols():
    build.build()
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True,
                         text=True).stdout
    syms = set(re.findall(r" T (dda_\w+)", out))
    assert set(_declared()) <= syms


def test_null_and_bad_arguments(L):
    assert L.dda_free(None) == dda.DDA_OK
    assert L.dda_build_Dmatrix(None, 0) == dda.DDA_ERR_ARG
    assert L.dda_matvec(None, 0, None, None, 1) == dda.DDA_ERR_ARG
    assert L.dda_last_error(None) == b"null handle"
    h = ctypes.c_void_p()
    occ = np.ones(8, dtype=np.uint8)
    m = np.array([1.5, 0.0])
    mp = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    op = occ.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    # invalid sizes, kd, material counts are rejected before any CUDA call
    assert L.dda_init_lattice(ctypes.byref(h), 0, 2, 2, op, 1, mp, 0.5, 0, None) == dda.DDA_ERR_ARG
    assert L.dda_init_lattice(ctypes.byref(h), 2, 2, 2, op, 1, mp, -1.0, 0, None) == dda.DDA_ERR_ARG
    assert L.dda_init_lattice(ctypes.byref(h), 2, 2, 2, op, 0, mp, 0.5, 0, None) == dda.DDA_ERR_ARG
    assert L.dda_init_lattice(None, 2, 2, 2, op, 1, mp, 0.5, 0, None) == dda.DDA_ERR_ARG
    assert h.value is None


def test_mueller_plane_host_logic(L):
    """S11 from the plane amplitudes equals the oracle's BH-matrix reading."""
    rng = np.random.default_rng(0)
    th = inputs.angles_deg(37)
    Fx = rng.standard_normal((37, 3)) + 1j * rng.standard_normal((37, 3))
    Fy = rng.standard_normal((37, 3)) + 1j * rng.standard_normal((37, 3))
    s11 = dda.dda_mueller_plane(th, Fx, Fy)
    ref = observables.s11_plane(Fx, Fy, th)
    assert np.allclose(s11, ref, rtol=1e-14, atol=0)


def test_mueller_full_host_logic(L):
    """All 16 elements from the closed forms equal the oracle's Mueller matrix
    by the Stokes-vector definition, on random amplitudes."""
    rng = np.random.default_rng(1)
    th = inputs.angles_deg(29)
    Fx = rng.standard_normal((29, 3)) + 1j * rng.standard_normal((29, 3))
    Fy = rng.standard_normal((29, 3)) + 1j * rng.standard_normal((29, 3))
    M = dda.dda_mueller_plane_full(th, Fx, Fy)
    ref = observables.mueller_plane(Fx, Fy, th)
    assert np.abs(M - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.allclose(M[:, 0, 0], dda.dda_mueller_plane(th, Fx, Fy), rtol=1e-14)


def test_asymmetry_host_logic(L):
    rng = np.random.default_rng(2)
    dirs, w = observables.sphere_quadrature(8, 12)
    F = rng.standard_normal((dirs.shape[0], 3)) + 1j * rng.standard_normal((dirs.shape[0], 3))
    a = np.array([0.6, 0.0, 0.8])
    g, gv = dda.dda_asymmetry(dirs, w, F, a)
    g0, gv0 = observables.asymmetry_from_farfield(F, dirs, w, a)
    assert abs(g - g0) < 1e-14 and np.allclose(gv, gv0, rtol=0, atol=1e-14)
    with pytest.raises(dda.DDAError):
        dda.dda_asymmetry(dirs, w, 0 * F, a)          # no scattered power
