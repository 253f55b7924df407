"""Waveform relaxation FAS for the 1-D nonlinear problem of Sec. 7 (oracle, test
infrastructure).

Problem (Eq. anomalous_diffusion) on (0,1) x (0,T], zero Dirichlet data and zero
initial value:
    D_t^delta u = d/dx( D(u) du/dx ) + c du/dx + f.
Discretisation at an interior point (x_n, t_m):
  * time: the L1 scheme (Eq. L1_scheme2); with u_0 = 0 it is the lower-triangular
    Toeplitz matrix T_M of Sec. 5 applied to the time line;
  * diffusion: the conservative flux difference of Eq. spatial_discretization,
        h^-2 [ a_{n+1/2,m} (u_{n+1,m} - u_{n,m}) - a_{n-1/2,m} (u_{n,m} - u_{n-1,m}) ],
        a_{n+-1/2,m} = ( D(u_{n+-1,m}) + D(u_{n,m}) ) / 2,
    with the boundary values 0 inside a at the first and last points;
  * convection: upwind.  For c >= 0 the term c u_x is carried by characteristics
    running towards smaller x, so its upwind difference is the forward one,
    c (u_{n+1,m} - u_{n,m}) / h; for c < 0 the backward one.
The discrete problem is N_h(u) = f with
    N_h(u) = T_M u_n - diffusion - convection       (every interior n, m).

Solver (Sec. 7, the paragraph after Eq. spatial_discretization): the full
approximation scheme (FAS) with a nonlinear red-black Gauss-Seidel waveform
smoother and the transfers of the linear method (full weighting, linear
interpolation; oracle.mgwr):
  * smoother: every point of one colour solves its own time line's equations
    with the neighbouring lines held fixed.  T_M is lower triangular, so that
    line system is solved step by step in time; at each step one scalar
    equation in u_{n,m}, which is strictly increasing for D(u) = 1 + u^2 (and
    for any constant D > 0), is solved by Newton's method to rounding level;
  * FAS cycle on level l (coarser levels are rediscretisations on 2h, 4h, ...):
        u <- S^nu1(u);  r = f - N_h(u);  ubar = R u;  f_c = N_2h(ubar) + R r;
        u_c = cycle on level l-1 from ubar with right-hand side f_c (gamma times);
        u <- u + P (u_c - ubar);  u <- S^nu2(u);
    on the one-point grid the line solve is exact;
  * stopping: max-norm of the defect reduced by `tol` from the initial iterate
    u = 0 (the zero initial condition), as in Table table_nonlinear.
The solution is restricted by full weighting too (the paper names only
"standard transfer-grid operators").

Fields are (n, M) arrays (n = 2^k - 1 interior points, column m at t_{m+1}).
"""
from __future__ import annotations

from typing import Callable

import numpy as np

from . import l1
from .mgwr import BLACK, ORDERS, RED, colour_mask, prolong_linear, restrict_fw

Coefficient = Callable[[np.ndarray], np.ndarray]


def porous_D(v: np.ndarray) -> np.ndarray:
    """D(u) = 1 + u^2 (Table table_nonlinear)."""
    return 1.0 + v * v


def porous_dD(v: np.ndarray) -> np.ndarray:
    return 2.0 * v


def constant_D(v: np.ndarray) -> np.ndarray:
    return np.ones_like(v)


def constant_dD(v: np.ndarray) -> np.ndarray:
    return np.zeros_like(v)


def _pad(u: np.ndarray) -> np.ndarray:
    """(n + 2, M) with the zero boundary rows."""
    out = np.zeros((u.shape[0] + 2, u.shape[1]))
    out[1:-1] = u
    return out


def spatial_term(u: np.ndarray, h: float, c: float, D: Coefficient) -> np.ndarray:
    """-(diffusion + convection) of Eq. spatial_discretization and the upwind
    difference at every interior point, for every time level."""
    w = _pad(u)
    Dw = D(w)
    a_plus = 0.5 * (Dw[2:] + Dw[1:-1])
    a_minus = 0.5 * (Dw[:-2] + Dw[1:-1])
    diffusion = (a_plus * (w[2:] - w[1:-1]) - a_minus * (w[1:-1] - w[:-2])) / (h * h)
    if c >= 0:
        convection = c * (w[2:] - w[1:-1]) / h
    else:
        convection = c * (w[1:-1] - w[:-2]) / h
    return -(diffusion + convection)


def operator(u: np.ndarray, Tm: np.ndarray, h: float, c: float, D: Coefficient) -> np.ndarray:
    """N_h(u): the L1 time term T_M u_n plus the spatial term, every interior point."""
    return u @ Tm.T + spatial_term(u, h, c, D)


def line_solve(u: np.ndarray, f: np.ndarray, rows: np.ndarray, Tm: np.ndarray, h: float,
               c: float, D: Coefficient, dD: Coefficient, max_newton: int = 100) -> None:
    """The nonlinear waveform step for the points `rows` (in place): each solves its
    time line's equations N_h(u)_{n,m} = f_{n,m}, m = 1..M, with its two neighbour
    lines fixed.  T_M is lower triangular, so step m has one unknown u_{n,m} once
    steps 1..m-1 are known; Newton's method solves that scalar equation
        g(v) = r_1 v + sum_{j<m} (T_M)_{mj} u_{n,j}
               - h^-2 [ (D(u_+) + D(v))/2 (u_+ - v) - (D(u_-) + D(v))/2 (v - u_-) ]
               - convection(v) - f_{n,m} = 0."""
    idx = np.flatnonzero(rows)
    if idx.size == 0:
        return
    w = _pad(u)
    up, um = w[idx + 2], w[idx]          # neighbour lines (zero beyond the boundary)
    Dp, Dm = D(up), D(um)
    fr = f[idx]
    r1 = Tm[0, 0]
    h2 = h * h
    lines = u[idx].copy()
    M = u.shape[1]
    for m in range(M):
        hist = lines[:, :m] @ Tm[m, :m]
        v = lines[:, m].copy()
        upm, umm = up[:, m], um[:, m]
        done = False
        for _ in range(max_newton):
            Dv, dDv = D(v), dD(v)
            diffusion = (0.5 * (Dp[:, m] + Dv) * (upm - v) - 0.5 * (Dm[:, m] + Dv) * (v - umm)) / h2
            convection = c * (upm - v) / h if c >= 0 else c * (v - umm) / h
            g = r1 * v + hist - diffusion - convection - fr[:, m]
            dg = (r1 + 0.5 * (Dp[:, m] + Dm[:, m] + 2.0 * Dv + dDv * (2.0 * v - upm - umm)) / h2
                  + abs(c) / h)
            step = g / dg
            v = v - step
            if done:
                break
            # converged (the step is at the rounding level of v or of the equation's
            # own terms): take one more step to settle
            scale = (np.abs(r1 * v) + np.abs(hist) + np.abs(diffusion) + np.abs(convection)
                     + np.abs(fr[:, m])) / dg
            done = bool(np.all(np.abs(step) <= 1e-13 * (np.abs(v) + scale) + 1e-300))
        else:
            raise RuntimeError("Newton's method did not converge in the line solve")
        lines[:, m] = v
    u[idx] = lines


def time_stepping(n: int, M: int, T: float, delta: float, f: np.ndarray, c: float = 1.0,
                  D: Coefficient = porous_D, dD: Coefficient = porous_dD,
                  max_newton: int = 100) -> np.ndarray:
    """The discrete solution by marching in time (not a relaxation): at each t_m,
    Newton's method on all n coupled equations of that step, with the tridiagonal
    Jacobian of the flux and upwind differences and banded solves."""
    import scipy.linalg as sla

    h = 1.0 / (n + 1)
    Tm = l1.toeplitz_matrix(delta, T, M)
    r1 = Tm[0, 0]
    u = np.zeros((n, M))
    for m in range(M):
        hist = u[:, :m] @ Tm[m, :m]
        v = u[:, m - 1].copy() if m else np.zeros(n)
        done = False
        for _ in range(max_newton):
            F = r1 * v + hist + spatial_term(v[:, None], h, c, D)[:, 0] - f[:, m]
            w = np.concatenate(([0.0], v, [0.0]))
            Dw, dDw = D(w), dD(w)
            a_plus = 0.5 * (Dw[2:] + Dw[1:-1])
            a_minus = 0.5 * (Dw[:-2] + Dw[1:-1])
            # derivatives of the flux difference (times h^2) w.r.t. u_n, u_{n+1}, u_{n-1}
            d_mid = 0.5 * dDw[1:-1] * (w[2:] - 2.0 * w[1:-1] + w[:-2]) - a_plus - a_minus
            d_up = 0.5 * dDw[2:] * (w[2:] - w[1:-1]) + a_plus
            d_dn = -0.5 * dDw[:-2] * (w[1:-1] - w[:-2]) + a_minus
            main = r1 - d_mid / (h * h)
            upper = -d_up / (h * h)
            lower = -d_dn / (h * h)
            if c >= 0:
                main += c / h
                upper -= c / h
            else:
                main -= c / h
                lower += c / h
            ab = np.zeros((3, n))
            ab[0, 1:] = upper[:-1]
            ab[1] = main
            ab[2, :-1] = lower[1:]
            step = sla.solve_banded((1, 1), ab, F)
            v = v - step
            if done:
                break
            scale = (np.abs(hist).max() + np.abs(f[:, m]).max()) / np.abs(main).max()
            done = bool(np.abs(step).max() <= 1e-13 * (np.abs(v).max() + scale) + 1e-300)
        else:
            raise RuntimeError("Newton's method did not converge in a time step")
        u[:, m] = v
    return u


class WRFAS:
    """Level hierarchy and FAS cycle for one nonlinear problem (n, M, T, delta, c, D)."""

    def __init__(self, n: int, M: int, T: float, delta: float, c: float = 1.0,
                 D: Coefficient = porous_D, dD: Coefficient = porous_dD, order: str = "text"):
        if n < 1 or (n + 1) & n:
            raise ValueError("n must be 2^k - 1")
        if order not in ORDERS:
            raise ValueError(order)
        self.n, self.M, self.T, self.delta, self.c = n, M, T, delta, c
        self.D, self.dD, self.order = D, dD, order
        self.Tm = l1.toeplitz_matrix(delta, T, M)
        sizes = [n]
        while sizes[-1] > 1:
            sizes.append((sizes[-1] - 1) // 2)
        self.sizes = sizes[::-1]  # coarsest first

    @property
    def finest(self) -> int:
        return len(self.sizes) - 1

    def h(self, l: int) -> float:
        return 1.0 / (self.sizes[l] + 1)

    def N(self, l: int, u: np.ndarray) -> np.ndarray:
        """N_h(u) on level l (rediscretised with that level's h)."""
        return operator(u, self.Tm, self.h(l), self.c, self.D)

    def defect(self, l: int, u: np.ndarray, f: np.ndarray) -> np.ndarray:
        return f - self.N(l, u)

    def sweep(self, l: int, u: np.ndarray, f: np.ndarray, colour: int) -> np.ndarray:
        """One colour half-sweep of the nonlinear waveform smoother (in place)."""
        rows = colour_mask(1, self.sizes[l], colour, self.order)
        line_solve(u, f, rows, self.Tm, self.h(l), self.c, self.D, self.dD)
        return u

    def smooth(self, l: int, u: np.ndarray, f: np.ndarray, steps: int) -> np.ndarray:
        for _ in range(steps):
            self.sweep(l, u, f, RED)
            self.sweep(l, u, f, BLACK)
        return u

    def cycle(self, l: int, u: np.ndarray, f: np.ndarray, nu1: int, nu2: int,
              gamma: int = 1) -> np.ndarray:
        """One FAS cycle at level l; returns the new iterate."""
        u = u.copy()
        if l == 0:
            line_solve(u, f, np.ones(self.sizes[0], bool), self.Tm, self.h(0), self.c,
                       self.D, self.dD)
            return u
        n = self.sizes[l]
        self.smooth(l, u, f, nu1)
        r = self.defect(l, u, f)
        ubar = restrict_fw(u, 1, n)
        fc = self.N(l - 1, ubar) + restrict_fw(r, 1, n)
        uc = ubar
        for _ in range(gamma):
            uc = self.cycle(l - 1, uc, fc, nu1, nu2, gamma)
        u += prolong_linear(uc - ubar, 1, self.sizes[l - 1])
        self.smooth(l, u, f, nu2)
        return u

    def solve(self, f: np.ndarray, nu1: int = 0, nu2: int = 1, gamma: int = 1,
              tol: float = 1e-10, max_cycles: int = 100, u0: np.ndarray | None = None):
        """Cycle from u0 (default 0) until ||f - N_h(u)||_inf <= tol ||f - N_h(u0)||_inf.

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
