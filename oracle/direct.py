"""The discrete solution of the fractional heat equation (oracle, test infrastructure).

1-D: Sec. 2, Eqs. (discrete_model_IVP_1)-(discrete_model_IVP_3); 2-D: Sec. 6,
Eqs. (discrete_model_IVP_2d_1)-(discrete_model_IVP_2d_3).  On the unit
interval / square with h = 1/(n+1):
    D_M u_{p,m} + (A_h u)_{p,m} = f_{p,m},   A_h = -Delta_h (3- or 5-point),
zero Dirichlet data and u_{p,0} = g_p.

``time_stepping`` is the plain definition: the system is block lower
triangular in time (Sec. 5: A = T_M (x) I_N + A_h), so it is solved step by
step; at step m the history sum is moved to the right-hand side and the
spatial system (r_1 I + A_h) u_m = rhs is solved by a sparse LU factorised once.
``dense_solve`` assembles the whole NM x NM matrix and solves it at once; it is
an independent route to the same vector for tiny grids.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import l1


def laplacian(d: int, n: int) -> sp.csr_matrix:
    """A_h = -Delta_h on n^d interior points, zero Dirichlet, p = i + n*j.

    1-D: (2u_i - u_{i-1} - u_{i+1}) / h^2, Sec. 2 Eq. (discrete_model_IVP_1).
    2-D: (4u - u_E - u_W - u_N - u_S) / h^2, Sec. 6 (Delta_h below the 2-D model).
    """
    h = 1.0 / (n + 1)
    one = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], shape=(n, n))
    if d == 1:
        A = one
    elif d == 2:
        I = sp.identity(n)
        A = sp.kron(I, one) + sp.kron(one, I)  # p = i + n*j: i is the fast index
    else:
        raise ValueError("d must be 1 or 2")
    return (A / (h * h)).tocsr()


def time_stepping(d: int, n: int, M: int, T: float, alpha: float,
                  f: np.ndarray, g: np.ndarray | None = None,
                  steps: int | None = None) -> np.ndarray:
    """Solve the discrete model by L1 time stepping; returns u of shape (N, M).

    ``steps`` (default M) limits the number of time levels computed, for
    bounded timing samples; the remaining columns are left at zero.
    """
    N = n ** d
    assert f.shape == (N, M)
    r = l1.toeplitz_column(alpha, T, M)
    dk = l1.l1_weights(alpha, M)
    c = l1.l1_scale(alpha, T, M)
    A = laplacian(d, n)
    lu = spla.splu((A + r[0] * sp.identity(N)).tocsc())
    steps = M if steps is None else steps
    # time-major work array: row m holds all points at t_{m+1}
    U = np.zeros((M, N))
    for m in range(steps):
        rhs = f[:, m].copy()
        if g is not None:
            rhs += c * dk[m + 1] * g  # -c d_m u_0 moved to the right-hand side
        if m > 0:
            # history sum_{k=1}^{m} r_{k+1} u_{m+1-k}  (1-based), i.e. r[k] * U[m-k]
            rhs -= r[1 : m + 1] @ U[m - 1 :: -1]
        U[m] = lu.solve(rhs)
    return np.ascontiguousarray(U.T)


def operator_dense(d: int, n: int, M: int, T: float, alpha: float) -> np.ndarray:
    """The whole space-time matrix I_N (x) T_M + A_h (x) I_M for the (N, M) layout."""
    N = n ** d
    Tm = l1.toeplitz_matrix(alpha, T, M)
    A = laplacian(d, n).toarray()
    return np.kron(np.eye(N), Tm) + np.kron(A, np.eye(M))


def dense_solve(d: int, n: int, M: int, T: float, alpha: float,
                f: np.ndarray, g: np.ndarray | None = None) -> np.ndarray:
    """All-at-once solve on tiny grids (library LU of the assembled matrix)."""
    N = n ** d
    rhs = f.astype(np.float64).copy()
    if g is not None:
        dk = l1.l1_weights(alpha, M)
        c = l1.l1_scale(alpha, T, M)
        rhs += c * np.outer(g, dk[1:])
    u = np.linalg.solve(operator_dense(d, n, M, T, alpha), rhs.reshape(-1))
    return u.reshape(N, M)


def apply_operator(d: int, n: int, M: int, T: float, alpha: float, u: np.ndarray) -> np.ndarray:
    """(T_M (x) I + A_h) u by direct sums: each line times T_M plus the stencil."""
    Tm = l1.toeplitz_matrix(alpha, T, M)
    return u @ Tm.T + laplacian(d, n) @ u
