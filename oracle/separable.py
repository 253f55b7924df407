"""Exact discrete solution for separable sources (oracle, test infrastructure).

If f_{p,m} = F_m phi_p with phi = prod sin(pi x_k) at the interior nodes, phi is
an eigenvector of the discrete Dirichlet operator A_h = -Delta_h (Sec. 2 /
Sec. 6 stencils) with eigenvalue
    lambda_h = (4 / h^2) * d * sin^2(pi h / 2),
so the discrete solution of T_M (x) I + A_h (Sec. 5) with zero initial data is
u_{p,m} = w_m phi_p with (T_M + lambda_h I) w = F: one M x M lower-triangular
solve instead of an N M^2 time-stepping run.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import l1


def eigenvalue(d: int, n: int) -> float:
    h = 1.0 / (n + 1)
    return d * 4.0 / (h * h) * math.sin(math.pi * h / 2.0) ** 2


# Largest M for which time_factor forms the dense M x M matrix (128 MiB).
DENSE_MAX_M = 4096


def time_factor_dense(d: int, n: int, M: int, T: float, alpha: float,
                      F: np.ndarray) -> np.ndarray:
    """w = (T_M + lambda_h I)^{-1} F by a dense triangular solve."""
    A = l1.toeplitz_matrix(alpha, T, M) + eigenvalue(d, n) * np.eye(M)
    return sla.solve_triangular(A, F, lower=True)


def time_factor_substitution(d: int, n: int, M: int, T: float, alpha: float,
                             F: np.ndarray) -> np.ndarray:
    """The same w by forward substitution on the Toeplitz column (Sec. 5 Eq.
    (Toeplitz_matrix): row m of T_M holds r_{m-j+1} in column j <= m), in O(M)
    memory and O(M^2) time, for M too long for the dense matrix:
        w_m = (F_m - sum_{j<m} a_{m-j} w_j) / a_0,  a = (r_1 + lambda_h, r_2, ..., r_M).
    """
    a = l1.toeplitz_column(alpha, T, M)
    a[0] += eigenvalue(d, n)
    ar = a[::-1].copy()  # ar[M-1-k] = a_k: row m's coefficients a_m..a_1 are ar[M-1-m : M-1]
    F = np.asarray(F, dtype=np.float64)
    w = np.zeros(M)
    for m in range(M):
        w[m] = (F[m] - np.dot(ar[M - 1 - m:M - 1], w[:m])) / a[0]
    return w


def time_factor(d: int, n: int, M: int, T: float, alpha: float, F: np.ndarray) -> np.ndarray:
    """w = (T_M + lambda_h I)^{-1} F: dense solve up to DENSE_MAX_M, forward
    substitution beyond."""
    if M <= DENSE_MAX_M:
        return time_factor_dense(d, n, M, T, alpha, F)
    return time_factor_substitution(d, n, M, T, alpha, F)


def solution(d: int, n: int, M: int, T: float, alpha: float, F: np.ndarray,
             phi: np.ndarray) -> np.ndarray:
    return np.outer(phi, time_factor(d, n, M, T, alpha, F))
