"""Mittag-Leffler function E_alpha(z) (oracle, test infrastructure).

Sec. 7, first experiment: with f = 0 and initial value g = sin x the continuous
solution of D^alpha u = u_xx is u = E_alpha(-t^alpha) sin x, where
    E_alpha(z) = sum_{k >= 0} z^k / Gamma(alpha k + 1)
is the Mittag-Leffler function (entire in z for alpha > 0).  On the scaled
problem of the tests the argument stays in [-1, 0], where the series needs at
most a few hundred terms, all bounded by max_k 1/Gamma(alpha k + 1) < 1.13, so
the alternating sum loses no digits to cancellation.  Written as that series
(terms through log-gamma).  Its rounding error is about 1e-16 times the sum of
the term magnitudes, E_alpha(|z|) <= exp(|z|^(1/alpha)) roughly, so the
evaluation is limited to |z|^(1/alpha) <= 8 and |z| <= 4.
"""
from __future__ import annotations

import math

import numpy as np

Z_MAX = 4.0     # |z| limit
ZPOW_MAX = 8.0  # limit on |z|^(1/alpha): term magnitudes stay below about e^8


def mittag_leffler(alpha: float, z) -> np.ndarray:
    """E_alpha(z) for real z (scalar or array), 0 < alpha <= 2, |z| <= Z_MAX."""
    if not (0.0 < alpha <= 2.0):
        raise ValueError("alpha must be in (0, 2]")
    z = np.asarray(z, dtype=np.float64)
    zmax = float(np.abs(z).max()) if z.size else 0.0
    if zmax > Z_MAX or zmax ** (1.0 / alpha) > ZPOW_MAX:
        raise ValueError("series evaluation only for |z| <= min(%g, %g^alpha)" % (Z_MAX, ZPOW_MAX))
    out = np.empty_like(z)
    for idx, x in np.ndenumerate(z):
        total = 0.0
        if x == 0.0:
            out[idx] = 1.0
            continue
        lx, sx = math.log(abs(x)), (-1.0 if x < 0 else 1.0)
        k = 0
        while True:
            term = math.exp(k * lx - math.lgamma(alpha * k + 1.0)) * (sx ** k)
            total += term
            # past the largest term the magnitudes decrease monotonically
            if k > 10 and abs(term) < 1e-18 * max(abs(total), 1e-300) and \
                    alpha * k + 1.0 > abs(x) ** (1.0 / alpha) + 2.0:
                break
            k += 1
            if k > 20000:
                raise RuntimeError("Mittag-Leffler series did not converge")
        out[idx] = total
    return out if out.ndim else float(out)
