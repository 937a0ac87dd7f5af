"""The double-float (hi + lo float pair) arithmetic of the FP64-class products,
emulated on the CPU with IEEE float32 operations, to pin the error claims the
GPU kernels rely on: a sum left unrenormalised represents the same value as
the renormalised one, and a chain of such sums followed by a product stays
within a small multiple of 2^-46 of the operands' magnitude, cancellation
included.  (The GPU operations themselves are checked against FP64 in
tests/native/df_check.cu.)  Products of two float32 are exact in float64, so
fl32(float64 arithmetic) gives the fused multiply-add of the device here."""
import numpy as np

F32 = np.float32


def split(v):
    hi = v.astype(F32)
    lo = (v - hi.astype(np.float64)).astype(F32)
    return hi, lo


def value(a):
    return a[0].astype(np.longdouble) + a[1].astype(np.longdouble)


def fma(x, y, z):
    return (x.astype(np.float64) * y.astype(np.float64) + z.astype(np.float64)).astype(F32)


def lazy_add(a, b):
    """two-sum of the high words, low words added to its error term, no renormalisation"""
    s = a[0] + b[0]
    bb = s - a[0]
    e = (a[0] - (s - bb)) + (b[0] - bb)
    return s, e + (a[1] + b[1])


def renorm_add(a, b):
    s, e = lazy_add(a, b)
    h = s + e
    return h, e - (h - s)


def mul(a, b):
    p = (a[0] * b[0]).astype(F32)
    e = fma(a[0], b[0], -p)
    e = fma(a[0], b[1], e)
    e = fma(a[1], b[0], e)
    h = p + e
    return h, e - (h - p)


def _inputs(rng, n, k, cancel):
    xs = [rng.standard_normal(n) for _ in range(k + 1)]
    if cancel:        # pairs that nearly cancel in the high words
        for j in range(1, k + 1, 2):
            xs[j] = -xs[j - 1] * (1 + 2.0 ** -20 * rng.standard_normal(n))
    return xs


def test_unrenormalised_sum_has_the_same_value():
    rng = np.random.default_rng(1)
    a, b = split(rng.standard_normal(100000)), split(rng.standard_normal(100000) * 1e-3)
    la, ra = lazy_add(a, b), renorm_add(a, b)
    assert np.array_equal(value(la), value(ra))


def test_sum_chains_then_product_within_bound():
    rng = np.random.default_rng(2)
    n = 20000
    for cancel in (False, True):
        for k in (1, 2, 4, 8):
            xs = _inputs(rng, n, k, cancel)
            y = rng.standard_normal(n)
            acc = split(xs[0])
            mag = np.abs(xs[0]).astype(np.longdouble)
            exact = xs[0].astype(np.longdouble)
            for j in range(1, k + 1):
                xj = split(xs[j])
                acc = lazy_add(acc, xj)
                exact = exact + value(xj)
                mag = mag + np.abs(xs[j])
            yd = split(y)
            prod = mul(acc, yd)
            ref = exact * value(yd)
            err = np.abs(value(prod) - ref) / (mag * np.abs(y))
            assert float(err.max()) < (k + 3) * 2.0 ** -46, (cancel, k, float(err.max()))


def test_low_word_stays_small_between_products():
    """after k unrenormalised sums the low word is at most a few ulp of the
    largest operand (it only collects the two-sum errors and the low words)"""
    rng = np.random.default_rng(3)
    n = 20000
    for k in (2, 8):
        xs = _inputs(rng, n, k, True)
        acc = split(xs[0])
        big = np.abs(xs[0])
        for j in range(1, k + 1):
            acc = lazy_add(acc, split(xs[j]))
            big = np.maximum(big, np.abs(xs[j]))
        ulp = np.spacing(big.astype(F32)).astype(np.float64)
        assert float((np.abs(acc[1]) / ulp).max()) <= 2 * k
