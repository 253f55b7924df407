"""L1 discretisation of the Caputo derivative (oracle, test infrastructure).

Sec. 2, Eq. (L1_scheme2): with tau = T/M,
    D_M u_m = c [ d_1 u_m - d_m u_0 + sum_{k=1}^{m-1} (d_{k+1} - d_k) u_{m-k} ],
    c = tau^{-alpha} / Gamma(2 - alpha),   d_k = k^{1-alpha} - (k-1)^{1-alpha}, k >= 1.
Sec. 5, Eq. (Toeplitz_matrix): the time part is the lower-triangular Toeplitz
matrix T_M with first column r_i = c (d_i - d_{i-1}), i = 1..M, d_0 = 0.

The paper gives d_k only as a difference of powers.  Evaluated that way it
loses about (k/alpha) ulps at large k, so d_k is evaluated here as
    d_k = (k-1)^beta * expm1(beta * log1p(1/(k-1))),  beta = 1 - alpha, k >= 2,
which is the same number written without the subtraction; d_1 = 1.
"""
from __future__ import annotations

import math

import numpy as np


def l1_scale(alpha: float, T: float, M: int) -> float:
    """c = tau^{-alpha} / Gamma(2 - alpha), Sec. 2 Eq. (L1_scheme2)."""
    tau = T / M
    return tau ** (-alpha) / math.gamma(2.0 - alpha)


def l1_weights(alpha: float, M: int) -> np.ndarray:
    """d_k for k = 0..M (d_0 = 0, d_1 = 1), Sec. 2 below Eq. (L1_scheme2)."""
    beta = 1.0 - alpha
    d = np.zeros(M + 1, dtype=np.float64)
    if M >= 1:
        d[1] = 1.0
    if M >= 2:
        km1 = np.arange(1, M, dtype=np.float64)  # k - 1 for k = 2..M
        d[2:] = km1 ** beta * np.expm1(beta * np.log1p(1.0 / km1))
    return d


def toeplitz_column(alpha: float, T: float, M: int) -> np.ndarray:
    """r_1..r_M of T_M (0-based array r[i-1] = r_i), Sec. 5 Eq. (Toeplitz_matrix)."""
    d = l1_weights(alpha, M)
    return l1_scale(alpha, T, M) * (d[1:] - d[:-1])


def toeplitz_matrix(alpha: float, T: float, M: int) -> np.ndarray:
    """Dense lower-triangular T_M (M x M); T[m, j] = r_{m-j+1} for j <= m."""
    r = toeplitz_column(alpha, T, M)
    Tm = np.zeros((M, M))
    for m in range(M):
        Tm[m, : m + 1] = r[m::-1]
    return Tm


def l1_derivative(u: np.ndarray, u0: float, alpha: float, T: float) -> np.ndarray:
    """Apply D_M to one time line u_1..u_M with initial value u_0.

    Written directly from Sec. 2 Eq. (L1_scheme2), term by term, as an
    independent check on T_M: D_M u = T_M u - c d_m u_0.
    """
    M = u.shape[0]
    d = l1_weights(alpha, M)
    c = l1_scale(alpha, T, M)
    out = np.zeros(M)
    for m in range(1, M + 1):
        s = d[1] * u[m - 1] - d[m] * u0
        for k in range(1, m):
            s += (d[k + 1] - d[k]) * u[m - k - 1]
        out[m - 1] = c * s
    return out
