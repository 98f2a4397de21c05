"""Error bounds of the arithmetic building blocks of the CUDA solvers (mtgp_selftest_arith), against
FP64 (and exact rational) references:

* the FP64 reciprocal of the per-frequency solvers: hardware approximation plus one third-order
  Householder step, within 2 ulp of 1/x;
* double-float (pairs of FP32 values) rounding of FP64 inputs within 2^-48, reciprocal (one
  Newton-Raphson step) within 2^-44, product, sum and x - y^2 within 2^-45 of the operands' scale;
* the double-float log-determinant accumulator (product over 32 values, one logarithm) within
  2^-40 of the FP64 sum of logarithms;
* the double-float kernel values: the order-2 DSI value 2^33 K exact, the SI values of smoothness 1-4
  within 2^-44 of K(0) against the Bernoulli polynomials evaluated exactly.
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


def _dsi_words(rng):
    X = [0, 1, 2, 3, 5, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, (1 << 32) - 1, 1 << 16, (1 << 16) - 1]
    X += [1 << k for k in range(32)]
    X += [int(v) for v in rng.integers(0, 1 << 32, size=2000, dtype=np.uint64)]
    X += [int(v) >> int(s) for v, s in zip(rng.integers(0, 1 << 32, size=2000, dtype=np.uint64),
                                            rng.integers(0, 32, size=2000))]
    return X


def test_dsi_kernel_value_exact():
    """2^33 K(X / 2^32) of the order-2 DSI kernel (Eq. 2.6) in double-float equals the integer
    3 2^32 - 2 b X - 5 2^(32 - b), b = -floor(log2(X / 2^32)) (3 2^32 at X = 0), exactly."""
    X = _dsi_words(np.random.default_rng(5))
    got = _run(7, np.array(X, dtype=np.float64))
    for x, g in zip(X, got):
        if x == 0:
            ref = 3 << 32
        else:
            b = 33 - x.bit_length()
            ref = (3 << 32) - 2 * b * x - 5 * (1 << (32 - b))
        assert g == float(ref), (x, g, ref)


def _bernoulli_poly(n, u):
    """B_n(u) exactly (Fractions): sum_k C(n, k) B_k u^(n - k) with the Bernoulli numbers B_k (B_1 = -1/2)."""
    from math import comb
    B = {0: Fraction(1), 1: Fraction(-1, 2), 2: Fraction(1, 6), 4: Fraction(-1, 30), 6: Fraction(1, 42),
         8: Fraction(-1, 30)}
    return sum(comb(n, k) * B.get(k, Fraction(0)) * u ** (n - k) for k in range(n + 1))


@pytest.mark.parametrize("alpha", [1, 2, 3, 4])
def test_si_kernel_value_double_float(alpha):
    """The SI kernel of smoothness alpha (Eq. 2.5), K(u) = (-1)^(alpha+1) (2 pi)^(2 alpha) / (2 alpha)! B_(2 alpha)(u),
    evaluated in double-float at u = X / 2^32: within 2^-44 of the kernel's scale K(0) of the exact value."""
    from math import factorial, pi
    rng = np.random.default_rng(alpha)
    X = [0, 1, (1 << 31) - 1, 1 << 31, (1 << 32) - 1] + [int(v) for v in rng.integers(0, 1 << 32, size=400, dtype=np.uint64)]
    got = _run(8, np.array(X, dtype=np.float64), np.full(len(X), float(alpha)))
    c = Fraction((-1) ** (alpha + 1)) * Fraction((2 * pi) ** (2 * alpha)) / factorial(2 * alpha)
    scale = abs(float(c * _bernoulli_poly(2 * alpha, Fraction(0))))
    for x, g in zip(X, got):
        ref = float(c * _bernoulli_poly(2 * alpha, Fraction(x, 1 << 32)))
        assert abs(g - ref) <= 2.0 ** -44 * scale, (alpha, x, g, ref)
