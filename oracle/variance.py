"""Polynomial control variate for the Hutchinson estimate (test infrastructure).

Sec. 3.1 names a "2-term polynomial" variance reduction for the trace
estimate but does not give the polynomial.  Reading: for a trace function f
and a polynomial p of degree d (d = 1: two terms, c0 + c1 x; optionally
d = 2) whose trace is known exactly,

    tr f(L) = tr (f - p)(L) + tr p(L),
    tr p(L) = c0 tr I + c1 tr L + c2 tr L^2,   tr L^2 = sum_ij L_ij^2,

and the stochastic estimate is taken of tr (f - p)(L) only.  The Gauss rule
of every probe is exact for polynomials of degree <= 2m - 1, so
sum_k tau_k^2 p(theta_k) = q_0^T p(L) q_0 exactly: the correction removes
the part of each probe's estimate that a degree-d polynomial explains,
without bias.  p is the Chebyshev interpolant of f of degree d on the
spectral interval [0, bound] (bound = 2 for the normalized Laplacian, 2 max d
for L = D - A), at the nodes (bound/2)(1 + cos(pi (j + 1/2) / (d + 1))).
"""
from __future__ import annotations

import numpy as np

from . import quadrature as _qd


def frobenius_sq(lap) -> float:
    """tr L^2 = sum_ij L_ij^2 of the Laplacian (its definition, summed over
    the stored entries)."""
    L = lap.matrix()
    return float(np.sum(np.asarray(L.multiply(L).sum())))


def chebyshev_coefficients(f, degree: int, bound: float) -> np.ndarray:
    """Monomial coefficients c_0..c_d of the degree-d interpolant of the
    scalar function f at the Chebyshev nodes of [0, bound]."""
    j = np.arange(degree + 1)
    x = 0.5 * bound * (1.0 + np.cos(np.pi * (j + 0.5) / (degree + 1)))
    V = np.vander(x, degree + 1, increasing=True)
    return np.linalg.solve(V, np.array([f(xi) for xi in x], dtype=np.float64))


def trace_cv(runs, n: int, f, degree: int, bound: float, tr_l: float, tr_l2: float):
    """Control-variate estimate of tr f(L) and its standard error from the
    probes' Gauss rules.  ``f`` is a scalar function of x."""
    c = chebyshev_coefficients(f, degree, bound)
    traces = np.array([n, tr_l, tr_l2][: degree + 1], dtype=np.float64)
    exact_part = float(np.dot(c, traces))

    def resid(th):
        th = np.asarray(th, dtype=np.float64)
        p = np.polynomial.polynomial.polyval(th, c)
        return np.vectorize(f)(th) - p

    per_probe = np.array([_qd.quadratic_form(r.theta, r.tau2, resid) for r in runs])
    mean, se = _qd.hutchinson(per_probe, n)
    return float(mean + exact_part), float(se)


def heat_trace_cv(runs, n: int, t, degree: int, bound: float, tr_l: float, tr_l2: float):
    """Heat trace h_t = tr exp(-t L) (Eq. heat-trace) with the control
    variate, for every t of the grid."""
    out, se = [], []
    for tv in np.asarray(t, dtype=np.float64):
        m, s = trace_cv(runs, n, lambda x, tv=tv: np.exp(-tv * x), degree, bound, tr_l, tr_l2)
        out.append(m)
        se.append(s)
    return np.array(out), np.array(se)
