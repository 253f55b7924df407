"""First column of (T_M + sigma I)^{-1} (oracle, test infrastructure).

Sec. 5 (smoothing procedure): every smoother step solves (T_M + sigma I) x = b
per spatial point, with sigma = 2d/h^2; the inverse of a lower-triangular
Toeplitz matrix is again lower-triangular Toeplitz, so its first column k
determines it and x = k * b (causal convolution truncated to M terms).

The paper computes k by divide and conquer; the plain definition is the
solution of (T_M + sigma I) k = e_1, obtained here by forward substitution.
"""
from __future__ import annotations

import numpy as np

from . import l1


def inverse_column_from_r(r: np.ndarray, sigma: float) -> np.ndarray:
    """Forward substitution for (T + sigma I) k = e_1, T with first column r."""
    M = r.shape[0]
    a = r.copy()
    a[0] += sigma
    k = np.zeros(M)
    k[0] = 1.0 / a[0]
    for m in range(1, M):
        # row m: sum_{j=0}^{m} a[m-j] k[j] = 0
        k[m] = -np.dot(a[m:0:-1], k[:m]) / a[0]
    return k


def inverse_column(alpha: float, T: float, M: int, sigma: float) -> np.ndarray:
    return inverse_column_from_r(l1.toeplitz_column(alpha, T, M), sigma)


def causal_apply(col: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y = L b for the lower-triangular Toeplitz L with first column ``col``.

    ``b`` may be (M,) or (P, M) (one line per row); direct O(M^2) sum.
    """
    M = col.shape[0]
    b2 = np.atleast_2d(b)
    y = np.zeros_like(b2)
    for m in range(M):
        y[:, m] = b2[:, : m + 1] @ col[m::-1]
    return y.reshape(b.shape)
