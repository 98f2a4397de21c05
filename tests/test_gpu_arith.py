"""Error bounds of the arithmetic building blocks of the CUDA solvers (mtgp_selftest_arith), against
FP64 (and exact rational) references:

* the FP64 reciprocal of the per-frequency solvers: hardware approximation plus one third-order
  Householder step, within 2 ulp of 1/x;
* double-float (pairs of FP32 values) rounding of FP64 inputs within 2^-48, reciprocal (one
  Newton-Raphson step) within 2^-44, product, sum and x - y^2 within 2^-45 of the operands' scale;
* the double-float log-determinant accumulator (product over 32 values, one logarithm) within
  2^-40 of the FP64 sum of logarithms.
"""
import ctypes
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_16014_gb300 import build
    build.build()


def _run(op, x, y=None):
    from paper_2603_16014_gb300._lib import check, lib
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yd = None if y is None else torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).cuda()
    out = torch.empty_like(xd)
    check(lib().mtgp_selftest_arith(op, xd.numel(), ctypes.c_void_p(xd.data_ptr()),
                                    ctypes.c_void_p(0 if yd is None else yd.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0)), "mtgp_selftest_arith")
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _values(rng, n, lo, hi, signed=False):
    x = np.exp2(rng.uniform(lo, hi, n)) * rng.uniform(1.0, 2.0, n)
    if signed:
        x *= np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    return x


def test_fp64_reciprocal_within_two_ulp():
    rng = np.random.default_rng(1)
    x = np.concatenate([_values(rng, 20000, -990, 990), [1.0, 2.0, 3.0, 1e-8, 1e8, 0.1, 7.0]])
    r = _run(0, x)
    # exact relative error on a sample through rationals, and the FP64-computed bound on all
    ulp = np.spacing(1.0 / x) / np.abs(1.0 / x)
    assert np.all(np.abs(r * x - 1.0) <= 2 * ulp + 2.0 ** -53)
    for xi, ri in zip(x[:200], r[:200]):
        assert abs(Fraction(ri) * Fraction(xi) - 1) <= Fraction(2, 2 ** 52)
    # outside the fast range: exact division
    big = np.array([2.0 ** 1010, 2.0 ** -1010 * 3.0])
    assert np.array_equal(_run(0, big), 1.0 / big)


def test_double_float_rounding_and_reciprocal():
    rng = np.random.default_rng(2)
    x = _values(rng, 20000, -100, 100, signed=True)
    back = _run(1, x)
    assert np.all(np.abs(back - x) <= 2.0 ** -48 * np.abs(x))
    xp = np.abs(x)
    r = _run(2, xp)
    assert np.all(np.abs(r * xp - 1.0) <= 2.0 ** -44)


def test_double_float_products_sums():
    rng = np.random.default_rng(3)
    x = _values(rng, 20000, -40, 40, signed=True)
    y = _values(rng, 20000, -20, 20, signed=True)
    p = _run(3, x, y)
    assert np.all(np.abs(p - x * y) <= 2.0 ** -45 * np.abs(x * y))
    s = _run(4, x, y)
    assert np.all(np.abs(s - (x + y)) <= 2.0 ** -45 * (np.abs(x) + np.abs(y)))
    # cancellation: y close to -x
    yc = -x * (1.0 + 2.0 ** -30 * rng.standard_normal(x.size))
    sc = _run(4, x, yc)
    assert np.all(np.abs(sc - (x + yc)) <= 2.0 ** -45 * (np.abs(x) + np.abs(yc)))
    f = _run(5, x, y)
    assert np.all(np.abs(f - (x - y * y)) <= 2.0 ** -44 * (np.abs(x) + y * y))


def test_double_float_log_product():
    rng = np.random.default_rng(4)
    x = _values(rng, 32 * 256, -60, 60)
    got = _run(6, x)[::32]
    ref = np.log(x).reshape(-1, 32).sum(axis=1)
    assert np.all(np.abs(got - ref) <= 2.0 ** -40 * np.maximum(np.abs(ref), 1.0) + 1e-12)
