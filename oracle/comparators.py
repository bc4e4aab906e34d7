"""The paper's O(m) comparators of Sec. 2.3 (test infrastructure).

Taylor expansion of the heat trace, Eq. hks-taylor (NetLSD's small-t
approximation):
    h_t ~ n - t tr L + (t^2 / 2) tr L^2,   tr L^2 = sum_ij L_ij^2.

The quadratic approximation of the VNGE (Eq. vnge-taylor, and FINGER's Q of
Chen et al. as printed in Sec. 2.3).  Reading: both printed forms are garbled
(the first sums tr L with tr L^2, the second squares tr D); the two-term
expansion -x ln x ~ x (1 - x), summed over the eigenvalues mu of P = L / tr L
(whose sum is 1), gives
    Q = 1 - tr(P^2) = 1 - tr(L^2) / tr(L)^2,
and tr(L^2) = sum_i d_i^2 + 2 sum_{i<j} w_ij^2 for L = D - A, the degree and
edge sums the printed FINGER form names.

FINGER-Hbar = -Q ln(2 max D / tr L) and FINGER-Hhat = -Q ln(lambda_max / tr L):
-Q ln(mu_max) with mu_max = lambda_max(P) either bounded by 2 max D / tr L
(the Gershgorin bound of L = D - A; 2 / tr L for the normalized Laplacian) or
estimated.  Reading: the printed denominator tr(L)^2 of the bar form is a
garble of tr(L) (the bound of lambda_max(P) is 2 max D / tr L).  lambda_max
here is given by the caller: the exact one, or the largest Ritz value of a
Lanczos run (which converges first).
"""
from __future__ import annotations

import math

import numpy as np

from . import variance as _var


def taylor_heat(lap, t) -> np.ndarray:
    """Eq. hks-taylor at every t."""
    t = np.asarray(t, dtype=np.float64)
    return lap.n - t * lap.trace + 0.5 * t * t * _var.frobenius_sq(lap)


def vnge_quadratic(lap) -> float:
    """Q = 1 - tr(L^2) / tr(L)^2 (0 for an empty Laplacian)."""
    if lap.trace <= 0:
        return 0.0
    return 1.0 - _var.frobenius_sq(lap) / lap.trace ** 2


def finger_bar(lap) -> float:
    """-Q ln(bound / tr L), bound = 2 (normalized) or 2 max D (combinatorial)."""
    if lap.trace <= 0:
        return 0.0
    return -vnge_quadratic(lap) * math.log(lap.norm_bound() / lap.trace)


def finger_hat(lap, lam_max: float) -> float:
    """-Q ln(lambda_max / tr L)."""
    if lap.trace <= 0 or lam_max <= 0:
        return 0.0
    return -vnge_quadratic(lap) * math.log(lam_max / lap.trace)


def relative_l2(approx, exact) -> float:
    """The relative l2 error of a descriptor against the exact one (Sec. 4.1)."""
    approx, exact = np.asarray(approx, dtype=np.float64), np.asarray(exact, dtype=np.float64)
    return float(np.linalg.norm(approx - exact) / np.linalg.norm(exact))
