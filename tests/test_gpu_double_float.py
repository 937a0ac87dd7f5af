"""Double-float arithmetic on the device (the FP32-refined form's residual
products and D-matrix build): every operation's error is a few units of
2^-46 relative to its operands, in the paired FP32 form and the scalar form
(a fused multiply-add contraction of the rounded product into the following
sum would show here as an error near 2^-24)."""
import os
import shutil
import subprocess

import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_double_float_operations(tmp_path):
    need_gpu()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "df_check")
    src = os.path.join(HERE, "native", "df_check.cu")
    inc = os.path.join(os.path.dirname(HERE), "paper_0704_0037_gb300", "csrc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "--expt-relaxed-constexpr", "-I", inc, "-o", exe, src], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    errs = {ln.split()[0]: float(ln.split()[1]) for ln in out.strip().splitlines()}
    assert set(errs) == {"add", "sub", "mul", "scale", "fmas", "add_scalar", "mul_scalar"}
    for name, e in errs.items():
        assert e < 2.0 ** -44, (name, e)
