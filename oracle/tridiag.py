"""Lowest eigenvalue of the Lanczos tridiagonal matrix T (Sec. 2.2).

T has a_1..a_m on the diagonal and b_2..b_m on both off-diagonals (Sec. 2.2, the matrix
T built from Algorithm 1's constants). The paper says its eigenvalues follow "by
standard methods"; the reading used here is Sturm-sequence bisection (the count of
negative pivots of the LDL^T factorisation of T - x I equals the number of eigenvalues
below x), iterated until the bracket cannot shrink in FP64.
"""
from __future__ import annotations

import numpy as np


def sturm_count(a: np.ndarray, b: np.ndarray, x: float) -> int:
    """Number of eigenvalues of T below x. a: diagonal (m), b: off-diagonal (m-1)."""
    count = 0
    d = 1.0
    tiny = np.finfo(np.float64).tiny
    for i in range(len(a)):
        off = b[i - 1] * b[i - 1] / d if i > 0 else 0.0
        d = (a[i] - x) - off
        if d == 0.0:
            d = -tiny
        if d < 0.0:
            count += 1
    return count


def lowest_eigenvalue(a, b) -> float:
    """lambda_min(T) by bisection on the Sturm count inside the Gershgorin interval."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = len(a)
    if m == 0:
        raise ValueError("empty T")
    rad = np.zeros(m)
    if m > 1:
        rad[:-1] += np.abs(b)
        rad[1:] += np.abs(b)
    lo = float(np.min(a - rad))
    hi = float(np.max(a + rad))
    span = max(abs(lo), abs(hi), 1e-300)
    lo -= 1e-15 * span + 1e-300
    hi += 1e-15 * span + 1e-300
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if sturm_count(a, b, mid) >= 1:
            hi = mid
        else:
            lo = mid
    return hi
