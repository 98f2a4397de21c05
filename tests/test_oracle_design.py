"""Pins for the oracle's design points and univariate kernels (CPU only).

Each check compares the oracle with something other than itself: values written out by
hand from a definition, a textbook series, an exact integral, or a structural property
that a wrong index, sign or dropped term would break.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import design

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_van_der_corput_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "van_der_corput.txt")) if not l.startswith("#")]
    for i, num, den in rows:
        v = design.van_der_corput_fixed(np.array([int(i)]))[0]
        assert Fraction(int(v), 1 << 32) == Fraction(int(num), int(den))


@pytest.mark.parametrize("m", [1, 3, 6, 9])
def test_lattice_is_permuted_grid(m):
    # Def. 2.1 with odd g: {v(i) g mod 1 : i < 2^m} is the grid {k / 2^m}
    rng = np.random.default_rng(m)
    g = 2 * rng.integers(0, 1 << 12, size=3) + 1
    X = design.lattice_points(g, np.zeros(3, dtype=np.uint32), 1 << m)
    for j in range(3):
        k = X[:, j].astype(np.uint64) >> np.uint64(32 - m)
        assert np.all((X[:, j].astype(np.uint64) & np.uint64((1 << (32 - m)) - 1)) == 0)
        assert sorted(k.tolist()) == list(range(1 << m))


def test_lattice_extensibility_and_shift():
    # Sec. 3.3: for 2^p > i, z_{2^p + i} = (z_{2^p} + z_i) mod 1; shift adds mod 1
    g = np.array([1, 433, 1021], dtype=np.uint32)
    sh = np.array([123456789, 4000000000, 7], dtype=np.uint32)
    Z = design.lattice_points(g, np.zeros(3, dtype=np.uint32), 64).astype(np.uint64)
    X = design.lattice_points(g, sh, 64).astype(np.uint64)
    for p in range(6):
        for i in range(1 << p):
            assert np.all(Z[(1 << p) + i] == (Z[1 << p] + Z[i]) % (1 << 32))
    assert np.all(X == (Z + sh.astype(np.uint64)) % (1 << 32))


def test_dnet_linearity_and_net_property():
    rng = np.random.default_rng(3)
    d, mm = 4, 10
    gen = np.zeros((d, mm), dtype=np.uint32)
    for j in range(d):
        for p in range(mm):
            w = 1 << (31 - p)
            for r in range(p):
                w |= int(rng.integers(0, 2)) << (31 - r)
            gen[j, p] = w
    Z = design.dnet_points(gen, np.zeros(d, dtype=np.uint32), 1 << mm).astype(np.uint64)
    # Sec. 3.3: z_{2^p + i} = z_{2^p} XOR z_i for 2^p > i
    for p in range(mm):
        for i in range(0, 1 << p, max(1, (1 << p) // 16)):
            assert np.all(Z[(1 << p) + i] == Z[1 << p] ^ Z[i])
    # an invertible m x m leading block puts one point in every interval [k/2^m, (k+1)/2^m)
    for m in range(1, mm + 1):
        k = Z[: 1 << m] >> np.uint64(32 - m)
        for j in range(d):
            assert sorted(k[:, j].tolist()) == list(range(1 << m))


# ------------------------------------------------------------------------------- SI kernel

@pytest.mark.parametrize("alpha", [1, 2, 3, 4])
def test_si_kernel_fourier_series(alpha):
    # Eq. 2.5 equals sum_{h != 0} e^{2 pi i h u} / |h|^{2 alpha} (Bernoulli polynomial Fourier series)
    u = np.array([0.0, 0.1, 0.25, 0.5, 0.73, 0.999])
    h = np.arange(1, 200001, dtype=np.float64)
    series = np.array([2.0 * np.sum(np.cos(2 * np.pi * h * x) / h ** (2 * alpha)) for x in u])
    tol = 2.0 / ((2 * alpha - 1) * 200000.0 ** (2 * alpha - 1)) + 1e-13
    assert np.allclose(design.si_kernel_1d(u, alpha), series, atol=tol, rtol=0)


def test_si_kernel_mean_zero_and_symmetric():
    xg, wg = np.polynomial.legendre.leggauss(20)
    u = 0.5 * (xg + 1)
    assert abs(0.5 * np.sum(wg * design.si_kernel_1d(u, 2))) < 1e-13      # int_0^1 K = 0 (Thm 'fast BC' premise)
    uu = np.linspace(0, 1, 33)
    assert np.allclose(design.si_kernel_1d(uu, 2), design.si_kernel_1d(1 - uu, 2), atol=1e-13)


@pytest.mark.parametrize("m", [3, 7, 10])
def test_si_lattice_grid_aliasing_closed_form(m):
    # on the grid u = k/n: K(k/n) = sum_f e^{2 pi i f k / n} A(f),
    # A(f) = n^-4 pi^4 (1 + 2 cos^2(pi f/n)) / (3 sin^4(pi f/n)) (f != 0), A(0) = pi^4 / (45 n^4)
    n = 1 << m
    f = np.arange(1, n)
    A = np.empty(n)
    A[0] = np.pi ** 4 / (45 * n ** 4)
    A[1:] = np.pi ** 4 * (1 + 2 * np.cos(np.pi * f / n) ** 2) / (3 * np.sin(np.pi * f / n) ** 4) / n ** 4
    k = np.arange(n)
    Kgrid = np.real(np.exp(2j * np.pi * np.outer(k, np.arange(n)) / n) @ A)
    X = (k.astype(np.uint64) << np.uint64(32 - m))
    got = design.kernel_1d("lattice", X, np.zeros_like(X))
    assert np.allclose(got, Kgrid, rtol=0, atol=1e-12 * max(1.0, np.abs(Kgrid).max()))


# ------------------------------------------------------------------------------ DSI kernel

def _mu2(k):
    bits = [p + 1 for p in range(64) if (k >> p) & 1][::-1]
    return sum(bits[:2])


@pytest.mark.parametrize("m", [1, 4, 8, 11])
def test_dsi_kernel_walsh_series_on_dyadic_grid(m):
    # The order-2 DSI kernel has the Walsh series K2(x) = sum_{k >= 1} 2^{-mu_2(k)} wal_k(x)
    # (mu_2(k) = a_1 + a_2 for k = 2^{a_1 - 1} + 2^{a_2 - 1} + ..., a_1 > a_2 > ...; the order-alpha
    # kernels of the higher-order digital-net literature cited in Sec. 2.2.2).  On x = i / 2^m the series
    # aliases exactly: K2(i/2^m) = sum_{f < 2^m} wal_f(i/2^m) A(f) with, summing k = f + 2^m j in closed form,
    # A(0) = 2^-m + 2^{-2m-1},  A(f) = 2^{-mu_2(f)} + 2^{-(m + bitlen f)} + 2^{-2m-1}.
    n = 1 << m
    A = np.empty(n)
    A[0] = 2.0 ** -m + 2.0 ** (-2 * m - 1)
    for f in range(1, n):
        A[f] = 2.0 ** -_mu2(f) + 2.0 ** -(m + f.bit_length()) + 2.0 ** (-2 * m - 1)
    i = np.arange(n)
    # wal_f(x) = (-1)^{sum_p f_p x_{p+1}}, digit x_{p+1} of i/2^m is bit m-1-p of i
    sgn = np.ones((n, n))
    for p in range(m):
        fp = (np.arange(n) >> p) & 1
        xp = (i >> (m - 1 - p)) & 1
        sgn *= 1 - 2 * np.outer(xp, fp)
    Kgrid = sgn @ A
    X = i.astype(np.uint64) << np.uint64(32 - m)
    got = design.kernel_1d("dnet", X, np.zeros_like(X))
    assert np.allclose(got, Kgrid, rtol=0, atol=1e-13)


def test_dsi_kernel_special_values_and_mean_zero():
    # beta(0) = t_1(0) = 0 gives K2(0) = 3/2 (Eq. 2.6 conventions); near 0 the kernel tends to 3/2
    X = np.array([0, 1, 2, 3, 1 << 31, 3 << 30, 1 << 30], dtype=np.uint64)
    K = design.dsi_kernel_1d(X)
    assert K[0] == 1.5
    assert abs(K[1] - 1.5) < 1e-7 and abs(K[2] - 1.5) < 1e-7
    # exact integral over [0,1): the kernel is affine on each [2^-b, 2^-b+1) (beta = b there)
    total = Fraction(0)
    for b in range(1, 200):
        lo, hi = Fraction(1, 2 ** b), Fraction(2, 2 ** b)
        c = Fraction(-1) + Fraction(5, 2) * (1 - Fraction(1, 2 ** b))
        total += c * (hi - lo) - Fraction(b, 2) * (hi * hi - lo * lo)
    assert abs(float(total)) < 1e-50
    # and the oracle's evaluation agrees with that affine form on each piece (midpoints)
    for b in range(1, 31):
        Xm = np.uint64(3 << (31 - b)) if b <= 30 else np.uint64(3)
        x = float(Xm) / 2 ** 32
        assert abs(design.dsi_kernel_1d(np.array([Xm]))[0] - (-1 - b * x + 2.5 * (1 - 2.0 ** -b))) < 1e-14


def test_product_kernel_form():
    # Eq. 2.4 with gamma = 1: product over coordinates of (1 + eta_j K)
    rng = np.random.default_rng(1)
    Xa = rng.integers(0, 1 << 32, size=(5, 3), dtype=np.uint64)
    Xb = rng.integers(0, 1 << 32, size=(5, 3), dtype=np.uint64)
    eta = np.array([0.3, 1.2, 0.7])
    for kind in ("lattice", "dnet"):
        q = design.product_kernel(kind, Xa, Xb, eta)
        ref = np.ones(5)
        for j in range(3):
            ref *= 1 + eta[j] * design.kernel_1d(kind, Xa[:, j], Xb[:, j])
        assert np.allclose(q, ref, rtol=1e-15)
        # symmetry K(x, x') = K(x', x)
        assert np.allclose(q, design.product_kernel(kind, Xb, Xa, eta), rtol=1e-14)
