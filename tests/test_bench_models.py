"""The algorithmic-byte models bench.py divides by the measured launch times
(the roofline's `achieved`): each pass's bytes written out from the pass
structure of the product, at the bench's 134^3 sphere on the 270^3 grid."""
import bench


def test_product_pass_bytes_134():
    n, M, n_occ = 134, 270, 1260552
    m = bench.kernel_models(n, M, n_occ)
    s = 8                                        # complex64
    b1 = 3 * M * n * n * s                       # [3][nz][ny][Mx]
    b2 = 3 * M * M * n * s                       # [3][nz][My][Mx]
    octant = 6 * (M // 2 + 1) ** 3 * s
    vec = 3 * n_occ * s
    assert m["p3_zconv_c64"]["bytes"] == 2 * b2 + octant == 589634688
    assert m["p2_yfft_c64"]["bytes"] == b1 + b2
    assert m["p4_yifft_c64"]["bytes"] == b2 + b1
    assert m["p1_xfft_c64"]["bytes"] > vec + b1       # plus the x index and material reads
    assert m["p5_xifft_c64"]["bytes"] > b1 + 2 * vec
    assert m["qmr_k1"]["bytes"] == 3 * vec and m["qmr_k2"]["bytes"] == 13 * vec
    for k in ("p1_xfft", "p2_yfft", "p3_zconv", "p4_yifft", "p5_xifft"):
        assert m[f"{k}_c64"]["bound"] == "hbm"
        assert m[f"{k}_df"]["bound"] == "alu"           # double-float: FP32-pipe arithmetic
    assert m["p3_zconv_df"]["bytes"] == 2 * m["p3_zconv_c64"]["bytes"]   # 16-byte elements


def test_dbuild_lines_model():
    n, M = 134, 270
    h = M // 2 + 1
    m = bench.kernel_models(n, M, 1)
    assert m["dbuild_lines"]["bytes"] == 2 * 3 * h * h * M * 16
