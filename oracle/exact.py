"""Exact determinant of a floating-point matrix by fraction-free (Bareiss) elimination.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every float64 entry is an integer times a power of two, so K * 2^E is an integer matrix
for a common E and det(K) = det(K 2^E) / 2^{E N} exactly.  Bareiss' one-step integer
elimination keeps every intermediate an exact integer (each division is exact).
"""
from __future__ import annotations

import math

import numpy as np


def _scale_exponent(A: np.ndarray) -> int:
    E = 0
    for x in A.ravel():
        x = float(x)
        if x == 0.0:
            continue
        num, den = x.as_integer_ratio()
        E = max(E, den.bit_length() - 1)
    return E


def exact_det_scaled(A: np.ndarray):
    """(D, E) with det(A) = D / 2^{E n}, D an exact Python integer."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    E = _scale_exponent(A)
    M = []
    for i in range(n):
        row = []
        for j in range(n):
            num, den = float(A[i, j]).as_integer_ratio()
            row.append(num * ((1 << E) // den))
        M.append(row)
    sign = 1
    prev = 1
    for k in range(n - 1):
        if M[k][k] == 0:
            piv = next((i for i in range(k + 1, n) if M[i][k] != 0), None)
            if piv is None:
                return 0, E
            M[k], M[piv] = M[piv], M[k]
            sign = -sign
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                M[i][j] = (M[i][j] * M[k][k] - M[i][k] * M[k][j]) // prev
            M[i][k] = 0
        prev = M[k][k]
    return sign * M[n - 1][n - 1], E


def exact_logdet(A: np.ndarray) -> float:
    """log det(A) for a matrix with positive determinant, from the exact integer determinant."""
    D, E = exact_det_scaled(A)
    if D <= 0:
        raise ValueError("determinant is not positive")
    n = np.asarray(A).shape[0]
    bl = D.bit_length()
    shift = max(bl - 60, 0)
    mant = D >> shift
    return math.log(mant) + (shift - E * n) * math.log(2.0)
