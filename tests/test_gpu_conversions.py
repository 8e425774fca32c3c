"""The precision conversions of the mixed-precision solver, bit for bit.

The defect correction hands the FP64 residual to the FP32 inner cycles as float(r * (1/s)) and adds
the correction back as fma(s, double(e), phi). With a power-of-two scale s the library evaluates
both with integer bit operations (rounding the significand to nearest even itself) instead of
FP64 instructions. These tests compare mg_op_scale_convert with the IEEE definitions computed on
the host: numpy's float64 multiply and round-to-nearest-even cast for the first, exact rational
arithmetic (fractions.Fraction, correctly rounded back to float64) for the fused multiply-add.
Inputs cover the cases where the bit manipulation could go wrong: ties at the 29 dropped bits
with even and odd kept bits, carries into the exponent, overflow to infinity, results below the
normal range (float subnormals), double subnormals, signed zeros, infinities and NaNs, and a
scale that is not a power of two (the plain formula).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _doubles_from_bits(hi, lo):
    return ((np.asarray(hi, np.uint64) << np.uint64(32)) | np.asarray(lo, np.uint64)).view(np.float64)


def _edge_doubles(rng, n_random):
    vals = [0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
            1e-310, np.finfo(np.float32).max, -np.finfo(np.float32).max, np.finfo(np.float32).tiny,
            float(np.finfo(np.float32).smallest_subnormal), 1e300, -1e-300]
    # significand patterns around the rounding point (29 dropped bits; tie = 0x10000000)
    for e in (1023, 1023 - 20, 1023 + 20, 1023 - 126, 1023 + 127, 1023 - 149, 1023 - 130):
        for mhi in (0x00000, 0x00001, 0xfffff, 0x12345, 0xffffe):
            for lo in (0x10000000, 0x30000000, 0x0fffffff, 0x10000001, 0xefffffff, 0xf0000000, 0xffffffff, 0):
                for sign in (0, 1):
                    hi = (sign << 31) | (e << 20) | mhi
                    vals.append(float(_doubles_from_bits([hi], [lo])[0]))
    x = np.array(vals, dtype=np.float64)
    # random magnitudes over a wide exponent range
    r = rng.standard_normal(n_random) * np.exp2(rng.integers(-160, 160, n_random).astype(np.float64))
    return np.concatenate([x, r])


def _edge_floats(rng, n):
    f32 = np.finfo(np.float32)
    base = np.array([0.0, -0.0, 1.0, -1.5, np.inf, -np.inf, f32.max, -f32.max, f32.tiny, f32.smallest_subnormal,
                     -f32.smallest_subnormal, 3e-39, 1e-30, 7.0e37], dtype=np.float32)
    r = (rng.standard_normal(n) * np.exp2(rng.integers(-140, 120, n).astype(np.float64))).astype(np.float32)
    return np.resize(np.concatenate([base, r]), n)


def _fma_exact(a: float, b: float, c: float) -> float:
    if not (np.isfinite(a) and np.isfinite(b)):
        return a * b + c  # an infinite or NaN product: IEEE rules of the sum
    if not np.isfinite(c):
        return c  # a finite product (however large) plus inf or NaN
    v = Fraction(a) * Fraction(b) + Fraction(c)
    if v == 0:
        # exact zero: +0 unless both the product and c are -0 (IEEE 754 sum of signed zeros)
        prod_neg = (np.signbit(a) != np.signbit(b))
        return -0.0 if (prod_neg and np.signbit(c) and a * b == 0 and c == 0) else 0.0
    try:
        return float(v)  # correctly rounded
    except OverflowError:
        return np.inf if v > 0 else -np.inf


def _same_bits(got, exp):
    got = np.asarray(got)
    exp = np.asarray(exp)
    nan = np.isnan(exp)
    assert np.array_equal(np.isnan(got), nan)
    ui = np.uint32 if got.dtype == np.float32 else np.uint64
    g = got.view(ui)[~nan]
    e = exp.view(ui)[~nan]
    bad = np.nonzero(g != e)[0]
    return bad


@pytest.mark.parametrize("sc", [1.0, 2.0 ** -40, 2.0 ** 37, 2.0 ** -126, 2.0 ** -900, 2.0 ** 1000, 0.3, 3.0e5])
def test_scale_convert_matches_ieee(sc):
    from paper_1410_6609_gb300.solver import scale_convert

    rng = np.random.default_rng(11)
    x = _edge_doubles(rng, 30000)
    n = x.size
    e = _edge_floats(rng, n)
    y = np.resize(_edge_doubles(np.random.default_rng(12), 100), n)
    y[: n // 2] = rng.standard_normal(n // 2) * sc  # comparable magnitudes: real cancellation

    xf, yo, xs = scale_convert(torch.from_numpy(x).cuda(), torch.from_numpy(e).cuda(), torch.from_numpy(y).cuda(), sc)
    xf = xf.cpu().numpy()
    yo = yo.cpu().numpy()
    xs = xs.cpu().numpy()

    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        xs_exp = x * sc
    bad = _same_bits(xs, xs_exp)
    assert bad.size == 0, f"x*s differs at {bad[:5]}: x={x[bad[:5]]}, got {xs[bad[:5]]}, want {xs_exp[bad[:5]]}"

    isc = 1.0 / sc
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        xf_exp = (x * isc).astype(np.float32)
    bad = _same_bits(xf, xf_exp)
    assert bad.size == 0, f"float(x/s) differs at {bad[:5]}: x={x[bad[:5]]}, got {xf[bad[:5]]}, want {xf_exp[bad[:5]]}"

    yo_exp = np.array([_fma_exact(sc, float(ei), float(yi)) for ei, yi in zip(e, y)], dtype=np.float64)
    bad = _same_bits(yo, yo_exp)
    assert bad.size == 0, (f"fma(s, e, y) differs at {bad[:5]}: e={e[bad[:5]]}, y={y[bad[:5]]}, "
                           f"got {yo[bad[:5]]}, want {yo_exp[bad[:5]]}")


def test_scale_convert_rejects_bad_arguments():
    from paper_1410_6609_gb300 import _lib

    lib = _lib.load()
    assert lib.mg_op_scale_convert(None, None, None, 4, 1.0, None, None, None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_op_scale_convert(None, None, None, -1, 1.0, None, None, None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_op_scale_convert(None, None, None, 0, 0.0, None, None, None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_op_scale_convert(None, None, None, 0, 1e-320, None, None, None, None) == _lib.MG_ERR_INVALID
    assert lib.mg_op_scale_convert(None, None, None, 0, 1.0, None, None, None, None) == _lib.MG_OK
