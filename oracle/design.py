"""Design points and univariate kernels, in 32-bit fixed point (value = X / 2^32).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Fixed point makes the shift mod 1 (Def. 2.1) and the digital XOR (Def. 2.2) exact;
points equal to 1 cannot occur, which settles the boundary remark of Sec. 2.2.1.
"""
from __future__ import annotations

from fractions import Fraction
from math import comb, factorial, pi

import numpy as np

TWO32 = 2.0 ** 32
MASK32 = (1 << 32) - 1


def van_der_corput_fixed(i: np.ndarray) -> np.ndarray:
    """v(i) = sum_p i_p 2^{-p-1} (Def. 2.1) as a 32-bit word: the bit reversal of i."""
    i = np.asarray(i, dtype=np.uint64)
    out = np.zeros_like(i)
    for p in range(32):
        out |= ((i >> np.uint64(p)) & np.uint64(1)) << np.uint64(31 - p)
    return out


def lattice_points(g: np.ndarray, shift: np.ndarray, n: int) -> np.ndarray:
    """Shifted rank-1 lattice in radical-inverse order (Def. 2.1).

    z_i = v(i) g mod 1, x_i = (z_i + Delta) mod 1, for i < n.  Returns (n, d) uint32.
    v(i) g mod 1 in fixed point is (v32(i) * g) mod 2^32 exactly, since v(i) = v32(i) / 2^32.
    """
    i = np.arange(n, dtype=np.uint64)
    v = van_der_corput_fixed(i)
    g = np.asarray(g, dtype=np.uint64)
    z = (v[:, None] * g[None, :]) & np.uint64(MASK32)
    x = (z + np.asarray(shift, dtype=np.uint64)[None, :]) & np.uint64(MASK32)
    return x.astype(np.uint32)


def dnet_points(gen_cols: np.ndarray, shift: np.ndarray, n: int) -> np.ndarray:
    """Digitally-shifted base-2 digital sequence in radical-inverse order (Def. 2.2).

    z_i = XOR_{p : i_p = 1} g_p, x_i = z_i XOR Delta, with gen_cols[j, p] the 32-bit word of
    column g_p in coordinate j.  Returns (n, d) uint32.
    """
    gen_cols = np.asarray(gen_cols, dtype=np.uint64)
    d, mm = gen_cols.shape
    if n > (1 << mm):
        raise ValueError("not enough generating-matrix columns")
    i = np.arange(n, dtype=np.uint64)
    z = np.zeros((n, d), dtype=np.uint64)
    for p in range(mm):
        bit = ((i >> np.uint64(p)) & np.uint64(1)).astype(bool)
        z[bit] ^= gen_cols[:, p][None, :]
    x = z ^ np.asarray(shift, dtype=np.uint64)[None, :]
    return x.astype(np.uint32)


def design_points(kind: str, gen, shift_t, n: int) -> np.ndarray:
    if kind == "lattice":
        return lattice_points(gen, shift_t, n)
    if kind == "dnet":
        return dnet_points(gen, shift_t, n)
    raise ValueError(kind)


# ---------------------------------------------------------------------------------------
# univariate kernels
# ---------------------------------------------------------------------------------------

def bernoulli_numbers(k: int) -> list:
    """B_0..B_k as exact fractions (B_1 = -1/2), from sum_{j<=m} C(m+1, j) B_j = 0."""
    B = [Fraction(1)]
    for mm in range(1, k + 1):
        B.append(-sum(comb(mm + 1, j) * B[j] for j in range(mm)) / (mm + 1))
    return B


def bernoulli_poly_coeffs(p: int) -> list:
    """Coefficients c_k of B_p(x) = sum_k c_k x^k: B_p(x) = sum_j C(p, j) B_j x^{p-j}."""
    B = bernoulli_numbers(p)
    c = [Fraction(0)] * (p + 1)
    for j in range(p + 1):
        c[p - j] += comb(p, j) * B[j]
    return c


def si_kernel_1d(u: np.ndarray, alpha: int = 2) -> np.ndarray:
    """Eq. 2.5: (-1)^{alpha+1} (2 pi)^{2 alpha} / (2 alpha)! * B_{2 alpha}(u), u = (x - x') mod 1."""
    c = bernoulli_poly_coeffs(2 * alpha)
    u = np.asarray(u, dtype=np.float64)
    poly = np.zeros_like(u)
    for k in range(2 * alpha, -1, -1):
        poly = poly * u + float(c[k])
    scale = (-1) ** (alpha + 1) * (2 * pi) ** (2 * alpha) / factorial(2 * alpha)
    return scale * poly


def dsi_beta_fixed(X: np.ndarray) -> np.ndarray:
    """beta(x) = -floor(log2 x) for x = X / 2^32 > 0, beta(0) = 0 (Eq. 2.6 conventions)."""
    X = np.asarray(X, dtype=np.uint64)
    bl = np.zeros(X.shape, dtype=np.int64)
    tmp = X.copy()
    for _ in range(33):
        nz = tmp > 0
        bl += nz
        tmp = tmp >> np.uint64(1)
    # floor(log2 X) = bit_length(X) - 1, floor(log2 x) = floor(log2 X) - 32
    return np.where(X > 0, 33 - bl, 0)


def dsi_kernel_1d(X: np.ndarray, alpha: int = 2) -> np.ndarray:
    """Eq. 2.6: the order-alpha term K_alpha(x) of the adaptive-smoothness DSI kernel, alpha = 1..4,
    with beta(x) = -floor(log2 x), t_nu(x) = 2^{-nu beta(x)} and beta(0) = t_nu(0) = 0:
      K_1 = 1/6 - t_1 / 2                                  (reading of the garbled printed alpha = 1 form:
                                                            the order-one Walsh kernel, mean zero)
      K_2 = -1 - beta x + 5/2 (1 - t_1)
      K_3 = -1 + beta x^2 - 5 (1 - t_1) x + 43/18 (1 - t_2)
      K_4 = -1 - 2/3 beta x^3 + 5 (1 - t_1) x^2 - 43/9 (1 - t_2) x + 701/294 (1 - t_3)
            + beta (1/48 sum_{a >= 1} (1 - 2 x_a) / 2^{3 (a - 1)} - 1/42),   x_a the binary digits of x.

    ``X`` is the fixed-point word of x = x_j XOR x'_j, so x has 32 digits and x_a = 0 for a > 32.
    """
    X = np.asarray(X, dtype=np.uint64)
    nz = X > 0
    beta = dsi_beta_fixed(X).astype(np.float64)
    x = X.astype(np.float64) / TWO32
    t1 = np.where(nz, np.exp2(-beta), 0.0)
    t2 = np.where(nz, np.exp2(-2.0 * beta), 0.0)
    t3 = np.where(nz, np.exp2(-3.0 * beta), 0.0)
    if alpha == 1:
        return 1.0 / 6.0 - 0.5 * t1
    if alpha == 2:
        return -1.0 - beta * x + 2.5 * (1.0 - t1)
    if alpha == 3:
        return -1.0 + beta * x ** 2 - 5.0 * (1.0 - t1) * x + 43.0 / 18.0 * (1.0 - t2)
    if alpha == 4:
        digit_sum = np.zeros(X.shape)
        for a in range(1, 33):
            x_a = ((X >> np.uint64(32 - a)) & np.uint64(1)).astype(np.float64)
            digit_sum += (1.0 - 2.0 * x_a) / 8.0 ** (a - 1)
        digit_sum += 8.0 ** -31 * 8.0 / 7.0            # digits 33, 34, ... are zero
        return (-1.0 - 2.0 / 3.0 * beta * x ** 3 + 5.0 * (1.0 - t1) * x ** 2 - 43.0 / 9.0 * (1.0 - t2) * x
                + 701.0 / 294.0 * (1.0 - t3) + beta * (digit_sum / 48.0 - 1.0 / 42.0))
    raise ValueError("DSI kernel order must be 1, 2, 3 or 4")


def dsi_mixture_1d(X: np.ndarray, b) -> np.ndarray:
    """Eq. 2.6: K(x, x') = sum_{alpha=1}^{4} b_alpha K_alpha(x XOR x'), weights b >= 0."""
    return sum(float(b[a - 1]) * dsi_kernel_1d(X, a) for a in range(1, 5) if b[a - 1] != 0.0)


def kernel_1d(kind: str, Xa: np.ndarray, Xb: np.ndarray, alpha=2) -> np.ndarray:
    """The univariate kernel of the kind's design/kernel pairing (Cond. 3.1) on fixed-point words.
    Lattices: alpha is the SI kernel's smoothness (Eq. 2.5).  Digital nets: alpha is either one order
    1..4 of Eq. 2.6 (weights b = e_alpha) or the four mixture weights b of Eq. 2.6."""
    Xa = np.asarray(Xa, dtype=np.uint64)
    Xb = np.asarray(Xb, dtype=np.uint64)
    if kind == "lattice":
        u = ((Xa - Xb) & np.uint64(MASK32)).astype(np.float64) / TWO32
        return si_kernel_1d(u, alpha)
    if kind == "dnet":
        if np.ndim(alpha) == 0:
            return dsi_kernel_1d(Xa ^ Xb, int(alpha))
        return dsi_mixture_1d(Xa ^ Xb, alpha)
    raise ValueError(kind)


def product_kernel(kind: str, Xa: np.ndarray, Xb: np.ndarray, eta: np.ndarray,
                   gamma: float = 1.0, alpha=2) -> np.ndarray:
    """Eq. 2.4: Q(x, x') = gamma prod_j (1 + eta_j K(x_j, x'_j)); Xa (..., d), Xb (..., d) broadcast."""
    Xa = np.asarray(Xa)
    Xb = np.asarray(Xb)
    out = None
    for j in range(len(eta)):
        f = 1.0 + eta[j] * kernel_1d(kind, Xa[..., j], Xb[..., j], alpha)
        out = f if out is None else out * f
    return gamma * out


def task_covariance(W: np.ndarray, v: np.ndarray) -> np.ndarray:
    """R = W W^T + diag(v) (Sec. 3.1, the paper's B B^T + diag(zeta))."""
    return W @ W.T + np.diag(v)
