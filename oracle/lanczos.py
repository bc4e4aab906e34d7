"""s-step Lanczos with full reorthogonalization (test infrastructure).

Sec. 3.1: from a unit starting vector q_0 the s-step Lanczos process builds an
orthonormal basis Q = [q_0 .. q_{s-1}] of the Krylov space
{q_0, L q_0, ..., L^{s-1} q_0} and the symmetric tridiagonal T = Q^T L Q
(diagonal alpha_k = q_k^T L q_k, off-diagonal beta_k), one matrix-vector
product with L per step (Algorithm 1, ``lanczos``).

Steps, per probe, in the order written here:
    w       = L q_k
    alpha_k = q_k^T w                                  (exactly rounded sum)
    w      -= alpha_k q_k + beta_{k-1} q_{k-1}          (three-term recurrence)
    w      -= Q (Q^T w)         once per reorthogonalization pass (classical
                                Gram-Schmidt against q_0..q_k; the paper does
                                not say how orthogonality is kept, one pass is
                                the default reading, two passes is CGS2)
    beta_k  = ||w||                                    (exactly rounded sum)
    q_{k+1} = w / beta_k

Breakdown (the paper is silent): if beta_k <= tol * bound, with bound the
Gershgorin bound of the spectrum (2 normalized, 2 max D combinatorial), the
Krylov space is exhausted and the probe's T is truncated to m = k+1.
The final step s-1 only needs alpha_{s-1}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DEFAULT_TOL = {"fp64": 1e-10, "fp32": 1e-4, "bf16": 1e-4}


@dataclass
class LanczosRun:
    alpha: np.ndarray   # float64[m]
    beta: np.ndarray    # float64[m-1]
    m: int
    Q: np.ndarray | None  # float64[n, m] (kept only when asked)


def _fsum_dot(a: np.ndarray, b: np.ndarray) -> float:
    return math.fsum((a * b).tolist())


def lanczos(L, v: np.ndarray, s: int, bound: float, reorth_passes: int = 1,
            tol: float = DEFAULT_TOL["fp64"], keep_basis: bool = False) -> LanczosRun:
    """Run s Lanczos steps of the sparse symmetric matrix ``L`` from ``v``."""
    if s < 1:
        raise ValueError("s must be >= 1")
    v = np.asarray(v, dtype=np.float64)
    nrm = math.sqrt(_fsum_dot(v, v))
    if nrm == 0.0:
        raise ValueError("zero starting vector")
    q = v / nrm
    basis = [q]
    alphas: list[float] = []
    betas: list[float] = []
    q_prev = None
    beta_prev = 0.0
    for k in range(s):
        w = L @ basis[k]
        alpha = _fsum_dot(basis[k], w)
        alphas.append(alpha)
        if k == s - 1:
            break
        w = w - alpha * basis[k]
        if q_prev is not None:
            w = w - beta_prev * q_prev
        Qm = np.column_stack(basis)
        for _ in range(reorth_passes):
            h = Qm.T @ w
            w = w - Qm @ h
        beta = math.sqrt(_fsum_dot(w, w))
        if beta <= tol * bound:
            break
        betas.append(beta)
        q_prev, beta_prev = basis[k], beta
        basis.append(w / beta)
    m = len(alphas)
    Q = np.column_stack(basis[:m]) if keep_basis else None
    return LanczosRun(alpha=np.asarray(alphas), beta=np.asarray(betas), m=m, Q=Q)
