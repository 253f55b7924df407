"""Seeded synthetic workloads for the time-fractional heat equation.

This module only builds inputs: grids, manufactured right-hand sides and
random fields.  It holds none of the solver's arithmetic (no L1 weights, no
Toeplitz operators, no smoother), so both the CUDA path and the CPU oracle may
import it.  It depends on numpy and the standard library only.

Layout of every space-time field (shape ``(N, M)``, C order):
  * ``N = n**d`` interior spatial points, ``p = i`` (1-D) or ``p = i + n*j``
    (2-D, ``i`` the x index, ``j`` the y index, both 0-based);
  * ``M`` time levels, column ``m`` holds time ``t_{m+1} = (m+1)*tau``,
    ``tau = T/M`` (the paper's uniform temporal mesh, Sec. 2).
Each row is one spatial point's whole time line, contiguous in memory.

Manufactured solutions (Sec. 7 uses ``t^2 sin sin``; the non-smooth
``t^alpha`` variant exercises the initial-layer regime discussed in Sec. 7):
  * ``u = t^2 * phi(x)``      with ``D^a t^2 = 2 t^(2-a) / Gamma(3-a)``
  * ``u = t^a * phi(x)``      with ``D^a t^a = Gamma(1+a)``
  * ``u = t * phi(x)``        with ``D^a t = t^(1-a) / Gamma(2-a)``
where ``phi(x) = prod_k sin(pi x_k)`` on (0,1)^d with zero Dirichlet data, so
``-Laplace u = d pi^2 u`` and ``f = (D^a w(t) + d pi^2 w(t)) phi(x)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SOLUTIONS = ("t2", "talpha", "t1")


def level_sizes(n: int) -> list[int]:
    """Interior points per dimension on every level, coarsest first.

    Spatial-only coarsening down to a single point (Sec. 3): n_l = 2 n_{l-1} + 1,
    n_0 = 1.  ``n`` must be of the form 2^k - 1.
    """
    if n < 1 or (n + 1) & n:
        raise ValueError(f"n must be 2^k - 1, got {n}")
    sizes = [n]
    while sizes[-1] > 1:
        sizes.append((sizes[-1] - 1) // 2)
    return sizes[::-1]


def interior_nodes(n: int) -> np.ndarray:
    """x_i = (i+1) h, i = 0..n-1, h = 1/(n+1) on the unit interval."""
    h = 1.0 / (n + 1)
    return (np.arange(n, dtype=np.float64) + 1.0) * h


def time_nodes(M: int, T: float) -> np.ndarray:
    """t_{m+1} = (m+1) tau for m = 0..M-1."""
    tau = T / M
    return (np.arange(M, dtype=np.float64) + 1.0) * tau


def phi(d: int, n: int) -> np.ndarray:
    """phi(x) = prod_k sin(pi x_k) at the interior nodes, flattened with p = i + n*j."""
    s = np.sin(math.pi * interior_nodes(n))
    if d == 1:
        return s.copy()
    if d == 2:
        # p = i + n*j  ->  row-major (j, i) flattening
        return np.outer(s, s).reshape(-1)
    raise ValueError("d must be 1 or 2")


def time_profile(kind: str, alpha: float, t: np.ndarray) -> np.ndarray:
    """w(t) of the exact solution u = w(t) phi(x)."""
    if kind == "t2":
        return t * t
    if kind == "talpha":
        return t ** alpha
    if kind == "t1":
        return t.copy()
    raise ValueError(kind)


def caputo_of_profile(kind: str, alpha: float, t: np.ndarray) -> np.ndarray:
    """Closed-form Caputo derivative D^alpha w(t) of the time profile."""
    if kind == "t2":
        return 2.0 * t ** (2.0 - alpha) / math.gamma(3.0 - alpha)
    if kind == "talpha":
        return np.full_like(t, math.gamma(1.0 + alpha))
    if kind == "t1":
        return t ** (1.0 - alpha) / math.gamma(2.0 - alpha)
    raise ValueError(kind)


@dataclass(frozen=True)
class Problem:
    d: int
    n: int
    M: int
    T: float
    alpha: float
    kind: str = "t2"

    @property
    def N(self) -> int:
        return self.n ** self.d

    @property
    def unknowns(self) -> int:
        return self.N * self.M

    def exact(self) -> np.ndarray:
        """Continuous solution sampled on the grid, shape (N, M)."""
        w = time_profile(self.kind, self.alpha, time_nodes(self.M, self.T))
        return np.outer(phi(self.d, self.n), w)

    def rhs_profile(self) -> np.ndarray:
        """F(t) with f = F(t) phi(x): D^a w + d pi^2 w."""
        t = time_nodes(self.M, self.T)
        return caputo_of_profile(self.kind, self.alpha, t) + self.d * math.pi ** 2 * time_profile(
            self.kind, self.alpha, t)

    def rhs(self, out: np.ndarray | None = None) -> np.ndarray:
        """Manufactured source f(x, t) on the grid, shape (N, M), float64 (into
        `out` when given, a C-contiguous (N, M) float64 array)."""
        if out is not None:
            return np.outer(phi(self.d, self.n), self.rhs_profile(), out=out)
        return np.ascontiguousarray(np.outer(phi(self.d, self.n), self.rhs_profile()))


def random_field(N: int, M: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform(-scale, scale) field of shape (N, M), reproducible from ``seed``."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(N, M))


def random_alphas(count: int, seed: int, lo: float = 0.1, hi: float = 0.9) -> np.ndarray:
    """Per-instance fractional orders alpha ~ U[lo, hi] (batched workload)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=count)


def request_stream(count: int = 2000, seed: int = 1608, rate: float = 1.0):
    """Served workload: a list of request dicts with Poisson arrival times.

    d by a fair coin; n = 2^k - 1 with k ~ U{5..12} (1-D) or U{5..9} (2-D);
    M = 2^j with j ~ U{7..12}; alpha ~ U[0.1, 0.9]; exact solution t^2 or
    t^alpha by a fair coin; inter-arrival times Exp(rate).
    """
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for r in range(count):
        d = 1 + int(rng.integers(0, 2))
        k = int(rng.integers(5, 13)) if d == 1 else int(rng.integers(5, 10))
        j = int(rng.integers(7, 13))
        alpha = float(rng.uniform(0.1, 0.9))
        kind = "t2" if rng.integers(0, 2) == 0 else "talpha"
        t += float(rng.exponential(1.0 / rate))
        out.append(dict(id=r, d=d, n=2 ** k - 1, M=2 ** j, alpha=alpha, kind=kind, arrival=t))
    return out
