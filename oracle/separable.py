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


def time_factor(d: int, n: int, M: int, T: float, alpha: float, F: np.ndarray) -> np.ndarray:
    """w = (T_M + lambda_h I)^{-1} F by a dense triangular solve."""
    A = l1.toeplitz_matrix(alpha, T, M) + eigenvalue(d, n) * np.eye(M)
    return sla.solve_triangular(A, F, lower=True)


def solution(d: int, n: int, M: int, T: float, alpha: float, F: np.ndarray,
             phi: np.ndarray) -> np.ndarray:
    return np.outer(phi, time_factor(d, n, M, T, alpha, F))
