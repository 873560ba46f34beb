"""Host-side check of the TF32-split bound the FP32-accurate tensor-core tests
use (tests/_parity.py: x3_unit).  TF32 keeps 10 fraction bits; hi = tf32(x)
and lo = tf32(x - hi) (round to nearest, ties away from zero, as cvt.rna.tf32
does) give |x - hi - lo| <= 2^-22 |x|, and the three products hi hi + hi lo +
lo hi miss x z by at most 3 2^-22 |x z| (the dropped lo lo and the two
splits).  Exact products of TF32 values fit a double, so the sums below are
exact but for FP64 rounding far below the bound."""
import numpy as np

from _parity import tf32_unit, x3_unit


def tf32_rna(x):
    """Round FP32 values to the TF32 grid (10 fraction bits), ties away from
    zero: add half a unit of the 13 dropped bits to the magnitude, clear them."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & ~np.uint64(0x1FFF)).astype(np.uint32)
    return b.view(np.float32)


def test_rounding_to_tf32_grid():
    x = np.array([1.0, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -11, 1.0 + 2.0 ** -12, -(1.0 + 2.0 ** -11), 3.0], np.float32)
    np.testing.assert_array_equal(tf32_rna(x), np.array([1.0, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -10, 1.0,
                                                         -(1.0 + 2.0 ** -10), 3.0], np.float32))


def test_split_error_within_bound_and_single_product_outside():
    rng = np.random.default_rng(7)
    for m in (8, 64, 256):
        X = rng.standard_normal((400, m)).astype(np.float32)
        Z = rng.standard_normal((300, m)).astype(np.float32)
        Z /= np.linalg.norm(Z, axis=1, keepdims=True)
        xh = tf32_rna(X); xl = tf32_rna(X - xh)
        zh = tf32_rna(Z); zl = tf32_rna(Z - zh)
        assert (np.abs(X.astype(np.float64) - xh - xl) <= 2.0 ** -22 * np.abs(X.astype(np.float64))).all()
        f = lambda a, b: a.astype(np.float64) @ b.astype(np.float64).T
        exact = f(X, Z)
        split = f(xh, zh) + f(xh, zl) + f(xl, zh)
        one = f(xh, zh)
        scale = np.abs(X.astype(np.float64)) @ np.abs(Z.astype(np.float64)).T
        assert (np.abs(split - exact) <= 3 * 2.0 ** -22 * scale).all()
        assert (np.abs(split - exact) <= x3_unit(m) * scale).all()
        # a single TF32 product (no lo terms) breaks the split's product bound
        # and errs about 2^10 times more than the split
        assert (np.abs(one - exact) > 3 * 2.0 ** -22 * scale).any()
        assert np.abs(one - exact).max() > 300 * np.abs(split - exact).max()


def test_single_tf32_product_within_its_own_bound_and_tight():
    """The single-product TF32 precision's bound (tests/_parity.py: tf32_unit):
    each operand rounded to 11 significant bits misses x z by at most
    (2 2^-11 + 2^-22) |x z|, so every correlation's error is within
    tf32_unit(m) sum_i |x_i z_i|; one operand pair, x = z = 1 + 2^-11 + 2^-13
    (rounded up to 1 + 2^-10), reaches 1.5 2^-11 of |x z|, so the bound's
    leading term 2 2^-11 is tight to a factor 4/3."""
    rng = np.random.default_rng(8)
    for m in (8, 64, 256):
        X = rng.standard_normal((400, m)).astype(np.float32)
        Z = rng.standard_normal((300, m)).astype(np.float32)
        Z /= np.linalg.norm(Z, axis=1, keepdims=True)
        f = lambda a, b: a.astype(np.float64) @ b.astype(np.float64).T
        err = np.abs(f(tf32_rna(X), tf32_rna(Z)) - f(X, Z))
        scale = np.abs(X.astype(np.float64)) @ np.abs(Z.astype(np.float64)).T
        assert (err <= tf32_unit(m) * scale).all()
    xs = np.float32(1.0 + 2.0 ** -11 + 2.0 ** -13)
    assert float(tf32_rna(np.array([xs]))[0]) == 1.0 + 2.0 ** -10
    p_err = abs(float(tf32_rna(np.array([xs]))[0]) ** 2 - float(xs) ** 2) / float(xs) ** 2
    assert 1.4 * 2.0 ** -11 < p_err <= 2 * 2.0 ** -11 + 2.0 ** -22
