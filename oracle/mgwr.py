"""Multigrid waveform relaxation, Algorithm 1 (oracle, test infrastructure).

Written from Sec. 3 (1-D) and Sec. 6 (2-D):
  * smoother: red-black Gauss-Seidel waveform relaxation, Eq. (red-black) /
    Eq. (red-black_2d).  The points visited first ("red") are, in the text,
    those with an even mesh index n (1-D) or even n+l (2-D); in the 0-based
    arrays used here that is odd i (1-D) and even i+j (2-D): order "text".
    The 1-D iteration counts of Table table_it_1d are reproduced only with the
    other 1-D order (odd n first, i.e. even i; order "table"), which is what
    an even array index gives when the array also holds the boundary node
    n = 0.  In 2-D both readings coincide.  Each visited point solves
    (T_M + 2d/h^2 I) u_p = f_p + h^-2 sum_{q neighbour of p} u_q
    for its whole time line (a dense triangular solve here; Sec. 5 does the
    same solve as a convolution with the inverse column);
  * defect r = f - (T_M (x) I + A_h) u (Algorithm 1, "Compute the defect");
  * full-weighting restriction and linear (1-D) / bilinear (2-D)
    interpolation applied to whole time lines (Sec. 3 and Sec. 6);
  * coarsening in space only down to one point (Sec. 3), rediscretised
    coarse operators, coarse problems with zero initial data, gamma = 1 (V)
    or 2 (W) recursive cycles, exact solve on the one-point grid.

Fields are (N, M) arrays, p = i + n*j, column m at t_{m+1}.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import l1
from .direct import laplacian

RED, BLACK = 0, 1


def grid(u: np.ndarray, d: int, n: int) -> np.ndarray:
    """View an (N, M) field as (n, M) or (n_y, n_x, M) (j slow, i fast)."""
    return u.reshape(n, -1) if d == 1 else u.reshape(n, n, -1)


ORDERS = ("text", "table")


def colour_mask(d: int, n: int, colour: int, order: str = "text") -> np.ndarray:
    """Boolean mask over p of the points of one colour (RED is swept first)."""
    if order not in ORDERS:
        raise ValueError(order)
    i = np.arange(n)
    if d == 1:
        red = (i % 2) == (1 if order == "text" else 0)
    else:
        ii, jj = np.meshgrid(i, i, indexing="xy")  # ii[j, i] = i, p = i + n*j
        red = ((ii + jj) % 2 == 0).reshape(-1)
    return red if colour == RED else ~red


def neighbour_sum(u: np.ndarray, d: int, n: int) -> np.ndarray:
    """sum of the 2d neighbour lines of every point, zero outside the grid."""
    g = grid(u, d, n)
    s = np.zeros_like(g)
    if d == 1:
        s[1:] += g[:-1]
        s[:-1] += g[1:]
    else:
        s[:, 1:] += g[:, :-1]
        s[:, :-1] += g[:, 1:]
        s[1:, :] += g[:-1, :]
        s[:-1, :] += g[1:, :]
    return s.reshape(u.shape)


def restrict_fw(r: np.ndarray, d: int, n: int) -> np.ndarray:
    """Full weighting: 1-D (1/4)[1 2 1]; 2-D its tensor product (1/16)[1 2 1]^T[1 2 1]."""
    nc = (n - 1) // 2
    g = grid(r, d, n)

    def fw1(a: np.ndarray, axis: int) -> np.ndarray:
        a = np.moveaxis(a, axis, 0)
        out = 0.25 * (a[0:-2:2] + 2.0 * a[1:-1:2] + a[2::2])
        return np.moveaxis(out, 0, axis)

    if d == 1:
        c = fw1(g, 0)
    else:
        c = fw1(fw1(g, 1), 0)
    return np.ascontiguousarray(c.reshape(nc ** d, -1))


def prolong_linear(e: np.ndarray, d: int, nc: int) -> np.ndarray:
    """Linear (1-D) / bilinear (2-D) interpolation to the fine grid n = 2nc+1.

    Fine point 2J+1 takes coarse value J; fine point 2J takes the mean of coarse
    J-1 and J, with zeros beyond the boundary.
    """
    n = 2 * nc + 1
    g = grid(e, d, nc)

    def lin1(a: np.ndarray, axis: int) -> np.ndarray:
        a = np.moveaxis(a, axis, 0)
        shape = (n,) + a.shape[1:]
        out = np.zeros(shape)
        out[1::2] = a
        out[0::2][1:] += 0.5 * a
        out[0::2][:-1] += 0.5 * a
        return np.moveaxis(out, 0, axis)

    if d == 1:
        f = lin1(g, 0)
    else:
        f = lin1(lin1(g, 1), 0)
    return np.ascontiguousarray(f.reshape(n ** d, -1))


@dataclass
class Level:
    n: int
    h: float
    sigma: float                 # 2d / h^2, the smoother's diagonal
    solve_matrix: np.ndarray     # T_M + sigma I (dense, lower triangular)
    A: object = field(repr=False)  # sparse A_h


class WRMG:
    """Level hierarchy and cycle of Algorithm 1 for one (d, n, M, T, alpha)."""

    def __init__(self, d: int, n: int, M: int, T: float, alpha: float, order: str = "text"):
        if n < 1 or (n + 1) & n:
            raise ValueError("n must be 2^k - 1")
        if order not in ORDERS:
            raise ValueError(order)
        self.d, self.n, self.M, self.T, self.alpha = d, n, M, T, alpha
        self.order = order
        self.Tm = l1.toeplitz_matrix(alpha, T, M)
        sizes = [n]
        while sizes[-1] > 1:
            sizes.append((sizes[-1] - 1) // 2)
        self.levels = []
        for nl in sizes[::-1]:  # coarsest first
            h = 1.0 / (nl + 1)
            sigma = 2.0 * d / (h * h)
            self.levels.append(Level(nl, h, sigma, self.Tm + sigma * np.eye(M), laplacian(d, nl)))

    @property
    def finest(self) -> int:
        return len(self.levels) - 1

    # --- components -----------------------------------------------------------------
    def sweep(self, l: int, u: np.ndarray, f: np.ndarray, colour: int) -> np.ndarray:
        """One colour half-sweep of the waveform smoother at level l (in place)."""
        lv = self.levels[l]
        mask = colour_mask(self.d, lv.n, colour, self.order)
        b = f[mask] + neighbour_sum(u, self.d, lv.n)[mask] / (lv.h * lv.h)
        u[mask] = sla.solve_triangular(lv.solve_matrix, b.T, lower=True).T
        return u

    def smooth(self, l: int, u: np.ndarray, f: np.ndarray, steps: int) -> np.ndarray:
        for _ in range(steps):
            self.sweep(l, u, f, RED)
            self.sweep(l, u, f, BLACK)
        return u

    def defect(self, l: int, u: np.ndarray, f: np.ndarray) -> np.ndarray:
        """r = f - (T_M (x) I + A_h) u, by direct sums."""
        lv = self.levels[l]
        return f - (u @ self.Tm.T + lv.A @ u)

    def coarsest_solve(self, f: np.ndarray) -> np.ndarray:
        """Exact solve on the one-point grid: (T_M + sigma_0) u = f."""
        lv = self.levels[0]
        return sla.solve_triangular(lv.solve_matrix, f.T, lower=True).T.copy()

    def cycle(self, l: int, u: np.ndarray, f: np.ndarray, nu1: int, nu2: int,
              gamma: int = 1) -> np.ndarray:
        """One WRMG cycle (Algorithm 1) at level l; returns the new iterate."""
        if l == 0:
            return self.coarsest_solve(f)
        u = u.copy()
        self.smooth(l, u, f, nu1)
        rc = restrict_fw(self.defect(l, u, f), self.d, self.levels[l].n)
        ec = np.zeros_like(rc)
        for _ in range(gamma):
            ec = self.cycle(l - 1, ec, rc, nu1, nu2, gamma)
        u += prolong_linear(ec, self.d, self.levels[l - 1].n)
        self.smooth(l, u, f, nu2)
        return u

    def solve(self, f: np.ndarray, nu1: int = 1, nu2: int = 1, gamma: int = 1,
              tol: float = 1e-10, max_cycles: int = 100, u0: np.ndarray | None = None):
        """Cycle from u0 (default 0) until ||f - A u||_inf <= tol ||f - A u0||_inf.

        Returns (u, history) with history[k] = ||r_k||_inf / ||r_0||_inf.
        """
        L = self.finest
        u = np.zeros_like(f) if u0 is None else u0.copy()
        r0 = np.abs(self.defect(L, u, f)).max()
        hist = [1.0]
        if r0 == 0.0:
            return u, hist
        for _ in range(max_cycles):
            u = self.cycle(L, u, f, nu1, nu2, gamma)
            hist.append(float(np.abs(self.defect(L, u, f)).max() / r0))
            if hist[-1] <= tol:
                break
        return u, hist
