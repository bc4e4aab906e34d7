"""Exact descriptors through a full eigendecomposition (test infrastructure).

The paper's ground truth (Sec. 2.3 and Sec. 4.1): compute the whole spectrum
and evaluate sum_i f(lambda_i) directly; O(n^3), small graphs only.
LAPACK's symmetric eigensolver (numpy.linalg.eigh / eigvalsh), as in Sec. 4.
"""
from __future__ import annotations

import numpy as np

from . import descriptors as _ds


def spectrum(lap) -> np.ndarray:
    return np.linalg.eigvalsh(lap.dense())


def heat_trace(lam, t) -> np.ndarray:
    return _ds.heat_f(t)(np.asarray(lam)).sum(axis=-1)


def wave_trace(lam, t):
    return _ds.wave_re_f(t)(np.asarray(lam)).sum(axis=-1), _ds.wave_im_f(t)(np.asarray(lam)).sum(axis=-1)


def vnge(lam, c: float) -> float:
    return float(_ds.vnge_f(c)(np.asarray(lam)).sum())


def quadratic_form(lap, v, f) -> np.ndarray:
    """q^T f(L) q for q = v/||v||, through the eigenvectors of L."""
    lam, phi = np.linalg.eigh(lap.dense())
    q = np.asarray(v, dtype=np.float64)
    q = q / np.linalg.norm(q)
    mu2 = (phi.T @ q) ** 2
    return np.sum(mu2 * f(lam), axis=-1)
