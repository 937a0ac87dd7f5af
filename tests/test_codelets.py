"""Host-side check of the register DFT codelets (csrc/codelets.cuh): every
length the fast product kernels compose, forward and inverse, in double and
float, against the DFT definition summed directly in long double."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0704_0037_gb300", "csrc")


def test_codelets_match_dft(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "codelet_check")
    src = os.path.join(ROOT, "tests", "native", "codelet_check.cu")
    subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-I", CSRC, "-x", "cu",
                    src, "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [r.split() for r in out if r.strip()]
    assert len(rows) == 22 * 4
    for n, prec, direction, err in rows:
        bound = 1e-14 if prec == "f64" else 4e-7
        assert float(err) < bound, (n, prec, direction, err)
