"""Semi-algebraic mode analysis of the 1-D two-grid waveform cycle (oracle, test
infrastructure; also a CPU tool: ``python -m oracle.sama``).

Sec. 4.1: Fourier analysis in space (infinite grid, modes e^{i theta x}), exact in
time.  Standard coarsening pairs each low frequency theta^0, |theta^0 h| <= pi/2,
with the high frequency theta^1 = theta^0 -+ pi/h (the 2h-harmonics); on the pair
every operator of the two-grid cycle is a 2 x 2 array of M x M lower-triangular
Toeplitz matrices (the L1 time operator of Sec. 5 plus a multiple of I_M):

  A_h(theta^a)   = T_M + Ahat(theta^a) I,  Ahat = (4/h^2) sin^2(theta h / 2)
  Jacobi symbol  = (T_M + Mhat I)^{-1} Nhat,  Mhat = 2/h^2, Nhat = Mhat - Ahat
  S_red, S_black = the red and black half-steps coupling the two harmonics
  C              = I_2M - P (T_M + A2hat I)^{-1} R A_h,  A2hat = (1/h^2) sin^2(theta^0 h)
  P, R           = linear interpolation / full weighting, (1 + cos theta^a h)/2 each
  T(theta^0)     = S^nu2 C S^nu1,  S = S_black S_red

and the predicted two-grid factor is the supremum of the spectral radius of
T(theta^0) over the low frequencies (Eq. two_grid_factor); Eq. smoothing_factor
takes the same supremum of the Jacobi symbol over the high frequencies.

All operators are scaled by h^2 (the factors do not change), so the time column
becomes r_i h^2 = (d_i - d_{i-1}) / lambda with lambda = tau^delta Gamma(2 - delta)
/ h^2 (Sec. 4.2), and the analysis depends only on (lambda, M, delta, theta h).

Readings taken here:
  * the symbol of h^-2 [-1 2 -1] is (4/h^2) sin^2(theta h / 2) (the square is lost
    in the printed formula);
  * the red points are the even fine points (those shared with the coarse grid),
    which is the coupling the printed S_red and S_black have; red goes first;
  * the coarse operator is the same stencil on 2h, and P and R have the symbols
    of linear interpolation and full weighting;
  * theta^1 = theta^0 - pi/h for theta^0 >= 0 (the printed sign(theta^0) is 0 at
    theta^0 = 0); only cos(theta^1 h) enters, so either choice gives the same T;
  * the supremum runs over theta^0 h = pi k / (2K), k = 1..K (the symbols are even
    in theta^0; theta^0 = 0 is left out because at lambda = inf its coarse symbol
    vanishes);
  * "spectral radius" is reported in two ways.  In exact arithmetic T(theta^0),
    reordered time step by time step, is block lower triangular with the same 2 x 2
    block on its diagonal, so its spectral radius is that block's and does not
    depend on M (mode "exact").  The factors the paper tabulates grow with M; the
    largest modulus among the eigenvalues that a dense double-precision
    nonsymmetric eigensolver (LAPACK's QR algorithm, numpy.linalg.eigvals) returns
    for T(theta^0) follows them (mode "dense").  T(theta^0) is far from normal,
    its eigenvalues are M-fold, and the computed ones scatter around the exact ones
    by about eps^(1/M) times the size of the strictly lower part: a rounding-driven
    (pseudospectral) value that depends on the eigensolver, most at small lambda.
    "exact" is the default of every function and of the command line; "dense" is
    kept as the explanation of the printed column's growth with M.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import l1


def lam_of(tau: float, h: float, delta: float) -> float:
    """lambda = tau^delta Gamma(2 - delta) / h^2 (Sec. 4.2)."""
    return tau ** delta * math.gamma(2.0 - delta) / (h * h)


def tau_of(lam: float, h: float, delta: float) -> float:
    """The time step that gives parameter `lam` on spatial step `h` (inverse of lam_of)."""
    return (lam * h * h / math.gamma(2.0 - delta)) ** (1.0 / delta)


def time_column(lam: float, M: int, delta: float) -> np.ndarray:
    """h^2 r_i, i = 1..M: the first column of h^2 T_M, r_i = c (d_i - d_{i-1}) (Sec. 5),
    c h^2 = 1 / lambda."""
    d = l1.l1_weights(delta, M)
    return (d[1:] - d[:-1]) / lam


def lower_toeplitz(col: np.ndarray) -> np.ndarray:
    """Dense lower-triangular Toeplitz matrix with first column `col`."""
    return np.tril(sla.toeplitz(col))


def harmonics(theta0: float) -> tuple[float, float]:
    """(theta^0 h, theta^1 h) for a low frequency theta^0 h in [-pi/2, pi/2] (Sec. 4.1)."""
    return theta0, (theta0 - math.pi if theta0 >= 0 else theta0 + math.pi)


def laplacian_symbol(theta: float) -> float:
    """h^2 Ahat(theta) for h^-2 [-1 2 -1]: 4 sin^2(theta h / 2)."""
    return 4.0 * math.sin(theta / 2.0) ** 2


def coarse_laplacian_symbol(theta0: float) -> float:
    """h^2 A2hat(theta^0): the same stencil on 2h seen by the coarse mode 2 theta^0."""
    return math.sin(theta0) ** 2


def transfer_symbol(theta: float) -> float:
    """Full weighting [1 2 1]/4 and linear interpolation: (1 + cos theta h) / 2."""
    return 0.5 * (1.0 + math.cos(theta))


def jacobi_symbol(lam: float, M: int, delta: float, theta: float) -> np.ndarray:
    """(T_M + Mhat I)^{-1} Nhat for one frequency (Sec. 4.1, Eq. algebraic_system):
    the point waveform Jacobi step, M_h the diagonal 2/h^2 of A_h."""
    col = time_column(lam, M, delta)
    col[0] += 2.0
    nhat = 2.0 - laplacian_symbol(theta)
    return nhat * sla.solve_triangular(lower_toeplitz(col), np.eye(M), lower=True)


def red_black_symbols(lam: float, M: int, delta: float, theta0: float):
    """(S_red, S_black), each 2M x 2M on the 2h-harmonics of theta^0 (Sec. 4.1)."""
    t0, t1 = harmonics(theta0)
    s0 = jacobi_symbol(lam, M, delta, t0)
    s1 = jacobi_symbol(lam, M, delta, t1)
    eye = np.eye(M)
    s_red = 0.5 * np.block([[s0 + eye, s1 - eye], [s0 - eye, s1 + eye]])
    s_black = 0.5 * np.block([[s0 + eye, eye - s1], [eye - s0, s1 + eye]])
    return s_red, s_black


def fine_operator_symbol(lam: float, M: int, delta: float, theta0: float) -> np.ndarray:
    """diag(T_M + Ahat(theta^0) I, T_M + Ahat(theta^1) I), 2M x 2M (Eq. fine_grid_operator_symbol)."""
    out = np.zeros((2 * M, 2 * M))
    for a, th in enumerate(harmonics(theta0)):
        col = time_column(lam, M, delta)
        col[0] += laplacian_symbol(th)
        out[a * M:(a + 1) * M, a * M:(a + 1) * M] = lower_toeplitz(col)
    return out


def coarse_grid_symbol(lam: float, M: int, delta: float, theta0: float) -> np.ndarray:
    """C = I_2M - P (T_M + A2hat I)^{-1} R A_h on the 2h-harmonics (Sec. 4.1)."""
    t0, t1 = harmonics(theta0)
    eye = np.eye(M)
    col = time_column(lam, M, delta)
    col[0] += coarse_laplacian_symbol(t0)
    coarse_inv = sla.solve_triangular(lower_toeplitz(col), eye, lower=True)
    R = np.hstack([transfer_symbol(t0) * eye, transfer_symbol(t1) * eye])
    P = np.vstack([transfer_symbol(t0) * eye, transfer_symbol(t1) * eye])
    return np.eye(2 * M) - P @ coarse_inv @ R @ fine_operator_symbol(lam, M, delta, theta0)


def two_grid_symbol(lam: float, M: int, delta: float, theta0: float,
                    nu1: int = 1, nu2: int = 0) -> np.ndarray:
    """T(theta^0) = S^nu2 C S^nu1, S = S_black S_red (Sec. 4.1, two-grid analysis)."""
    s_red, s_black = red_black_symbols(lam, M, delta, theta0)
    S = s_black @ s_red
    C = coarse_grid_symbol(lam, M, delta, theta0)
    return np.linalg.matrix_power(S, nu2) @ C @ np.linalg.matrix_power(S, nu1)


def spectral_radius(A: np.ndarray, blocks: int, mode: str = "exact") -> float:
    """Spectral radius of a blocks x blocks array of M x M lower-triangular Toeplitz
    matrices: "dense" = largest |eigenvalue| from the dense nonsymmetric eigensolver;
    "exact" = that of the blocks x blocks matrix of the blocks' diagonals."""
    M = A.shape[0] // blocks
    if mode == "dense":
        return float(np.abs(np.linalg.eigvals(A)).max())
    if mode == "exact":
        diag = A[::M, ::M]
        return float(np.abs(np.linalg.eigvals(diag)).max())
    raise ValueError(f"unknown mode {mode!r}")


def low_frequencies(K: int) -> np.ndarray:
    """theta^0 h = pi k / (2K), k = 1..K."""
    return math.pi * np.arange(1, K + 1) / (2.0 * K)


def high_frequencies(K: int) -> np.ndarray:
    """theta h = pi/2 + pi k / (2K), k = 1..K (the high frequencies, up to sign)."""
    return math.pi / 2.0 + math.pi * np.arange(1, K + 1) / (2.0 * K)


def two_grid_factor(lam: float, M: int, delta: float, nu1: int = 1, nu2: int = 0,
                    K: int = 64, mode: str = "exact") -> float:
    """Predicted two-grid factor rho = sup over theta^0 of rho(T(theta^0)) (Eq. two_grid_factor).
    In mode "exact" only the first time step enters (the diagonal of a product of
    lower-triangular matrices is the product of their diagonals), so M = 1 is used."""
    Mx = 1 if mode == "exact" else M
    return max(spectral_radius(two_grid_symbol(lam, Mx, delta, t, nu1, nu2), 2, mode)
               for t in low_frequencies(K))


def smoothing_factor(lam: float, M: int, delta: float, K: int = 64,
                     mode: str = "exact") -> float:
    """mu = sup over high frequencies of rho(Jacobi symbol) (Eq. smoothing_factor)."""
    Mx = 1 if mode == "exact" else M
    return max(spectral_radius(jacobi_symbol(lam, Mx, delta, t), 1, mode)
               for t in high_frequencies(K))


def _main(argv=None) -> None:
    import argparse
    ap = argparse.ArgumentParser(description="Two-grid factors predicted by semi-algebraic "
                                 "mode analysis (1-D, red-black waveform smoother, L1 scheme)")
    ap.add_argument("--delta", type=float, default=0.4, help="fractional order")
    ap.add_argument("--log2lam", default="-8:8:2", help="lo:hi:step of log2(lambda); write --log2lam=-8:8:2")
    ap.add_argument("--M", default="32,64,128", help="comma-separated time-step counts")
    ap.add_argument("--nu", default="1,0", help="pre,post smoothing steps")
    ap.add_argument("--K", type=int, default=64, help="low frequencies sampled")
    ap.add_argument("--mode", choices=("dense", "exact"), default="exact",
                    help="exact: the M-independent spectral radius (default); dense: the "
                         "largest modulus a dense eigensolver returns, which follows the "
                         "M-growth of the paper's predicted column")
    a = ap.parse_args(argv)
    lo, hi, step = (int(x) for x in a.log2lam.split(":"))
    Ms = [int(x) for x in a.M.split(",")]
    nu1, nu2 = (int(x) for x in a.nu.split(","))
    try:  # small eigenproblems: one BLAS thread is the fastest
        from threadpoolctl import threadpool_limits
        limit = threadpool_limits(1)
    except ImportError:
        limit = None
    print("log2_lambda " + " ".join(f"M={M:<6d}" for M in Ms))
    for e in range(lo, hi + 1, step):
        vals = [two_grid_factor(2.0 ** e, M, a.delta, nu1, nu2, a.K, a.mode) for M in Ms]
        print(f"{e:11d} " + " ".join(f"{v:<8.4f}" for v in vals), flush=True)
    if limit is not None:
        limit.restore_original_limits()


if __name__ == "__main__":
    _main()
