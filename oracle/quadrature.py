"""Gauss quadrature from the Lanczos tridiagonal (test infrastructure).

Eq. quadratic (Sec. 3.1): with T = U Lambda U^T, the m-point Gauss rule for
v^T f(L) v (unit v) has nodes theta_k = Lambda_kk (the eigenvalues of T) and
weights tau_k^2 with tau_k = U_{0,k}, the first component of the k-th
normalized eigenvector (Golub-Welsch).  Algorithm 1, ``slq``: eigh(T), then
sum_k f(theta_k) tau_k^2.

Eq. slq: over n_v probes the Hutchinson estimate of tr f(L) is
(n / n_v) sum_i sum_k (tau_k^i)^2 f(theta_k^i), with n the node count (n').
Algorithm 1 prints 1/n_v instead of n/n_v; with unit q_0 = v / ||v|| only
n/n_v is unbiased (h_0 = n exactly), which is the reading used.
The standard error of the mean is std_p(g_p) / sqrt(n_v) (ddof = 1).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh_tridiagonal


def ritz(alpha: np.ndarray, beta: np.ndarray):
    """Nodes theta (ascending) and weights tau^2 of the Gauss rule of T."""
    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    m = alpha.size
    if m == 1:
        return alpha.copy(), np.ones(1)
    theta, U = eigh_tridiagonal(alpha, beta)
    return theta, U[0, :] ** 2


def quadratic_form(theta, tau2, f) -> np.ndarray:
    """sum_k tau_k^2 f(theta_k); ``f`` maps theta -> values (broadcasting)."""
    return np.sum(np.asarray(tau2) * f(np.asarray(theta)), axis=-1)


def hutchinson(per_probe: np.ndarray, n: int):
    """Mean and standard error over probes of n * per_probe (axis 0)."""
    g = n * np.asarray(per_probe, dtype=np.float64)
    nv = g.shape[0]
    mean = g.sum(axis=0) / nv
    if nv > 1:
        se = np.sqrt(((g - mean) ** 2).sum(axis=0) / (nv - 1) / nv)
    else:
        se = np.full_like(mean, np.nan)
    return mean, se
