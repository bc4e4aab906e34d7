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


def _omega_next(alphas, betas, om_cur, om_prev, beta, eps):
    """omega_{k+1, 0..k+1} from omega_{k, .} (om_cur) and omega_{k-1, .}
    (om_prev), with alphas = alpha_0..alpha_k, betas = beta_0..beta_{k-1}
    and beta = beta_k (the recurrence of ``lanczos_partial``)."""
    k = len(alphas) - 1
    out = [0.0] * (k + 2)
    for j in range(k):
        t = betas[j] * om_cur[j + 1] + (alphas[j] - alphas[k]) * om_cur[j]
        if j > 0:
            t += betas[j - 1] * om_cur[j - 1]
        if k > 0:
            t -= betas[k - 1] * om_prev[j]
        t += math.copysign(eps * (beta + betas[j]), t)
        out[j] = t / beta if beta > 0.0 else math.inf
    out[k] = eps
    out[k + 1] = 1.0
    return out


@dataclass
class PartialRun(LanczosRun):
    full_steps: list    # steps k whose new vector q_{k+1} was reorthogonalized
    omega_max: list     # per step k: max_j |omega_{k+1,j}| before any reorthogonalization


def lanczos_partial(L, v: np.ndarray, s: int, bound: float, eps: float = 2.0 ** -53,
                    tol: float = DEFAULT_TOL["fp64"], keep_basis: bool = False) -> PartialRun:
    """s Lanczos steps with partial reorthogonalization (not in the paper).

    Simon (Math. Comp. 42, 1984): the three-term recurrence alone loses
    orthogonality as Ritz values converge, but it is enough that the basis
    stays semi-orthogonal, |q_i^T q_j| <= sqrt(eps), for T to be the
    projection of L to working accuracy.  The level omega_{k,j} ~ q_k^T q_j is
    estimated at no cost by the recurrence that q_k^T L q_j = q_j^T L q_k
    imposes on it; for the new vector q_{k+1} and j < k,

        beta_k omega_{k+1,j} = beta_j omega_{k,j+1} + (alpha_j - alpha_k) omega_{k,j}
                               + beta_{j-1} omega_{k,j-1} - beta_{k-1} omega_{k-1,j}

    (omega_{i,i} = 1, terms with negative indices vanish), plus a rounding
    term eps (beta_k + beta_j) taken in the direction that grows |omega|.
    omega_{k+1,k} is the local level eps.  When max_j |omega_{k+1,j}| exceeds
    sqrt(eps) the new vector is orthogonalized against all previous ones (one
    classical Gram-Schmidt pass), and so is the one after it, since the
    recurrence for q_{k+2} still carries the error of q_k; the estimates of
    a reorthogonalized vector are reset to eps.  Steps, per probe, in order:
        w = L q_k;  alpha_k = q_k^T w;  w -= alpha_k q_k + beta_{k-1} q_{k-1}
        beta_k = ||w||;  omega_{k+1, .} by the recurrence
        if forced or max |omega_{k+1,j}| > sqrt(eps): w -= Q (Q^T w), beta_k = ||w||
        breakdown test on beta_k (as in ``lanczos``);  q_{k+1} = w / beta_k
    ``eps`` is the unit roundoff of the arithmetic whose orthogonality is
    tracked (2^-53 here; 2^-24 for an FP32 basis)."""
    if s < 1:
        raise ValueError("s must be >= 1")
    v = np.asarray(v, dtype=np.float64)
    nrm = math.sqrt(_fsum_dot(v, v))
    if nrm == 0.0:
        raise ValueError("zero starting vector")
    basis = [v / nrm]
    alphas: list[float] = []
    betas: list[float] = []
    thr = math.sqrt(eps)
    om_prev: list[float] = []        # omega_{k-1, 0..k-1}
    om_cur: list[float] = [1.0]      # omega_{k, 0..k}
    force = False
    full_steps: list[int] = []
    omega_max: list[float] = []
    for k in range(s):
        w = L @ basis[k]
        alpha = _fsum_dot(basis[k], w)
        alphas.append(alpha)
        if k == s - 1:
            break
        w = w - alpha * basis[k]
        if k > 0:
            w = w - betas[k - 1] * basis[k - 1]
        beta = math.sqrt(_fsum_dot(w, w))
        om_next = _omega_next(alphas, betas, om_cur, om_prev, beta, eps)
        worst = max((abs(x) for x in om_next[:k]), default=0.0)
        omega_max.append(worst)
        triggered = worst > thr
        if force or triggered:
            Qm = np.column_stack(basis)
            w = w - Qm @ (Qm.T @ w)
            beta = math.sqrt(_fsum_dot(w, w))
            for j in range(k + 1):
                om_next[j] = eps
            full_steps.append(k)
        force = triggered and not force
        if beta <= tol * bound:
            break
        betas.append(beta)
        basis.append(w / beta)
        om_prev, om_cur = om_cur, om_next
    m = len(alphas)
    Q = np.column_stack(basis[:m]) if keep_basis else None
    return PartialRun(alpha=np.asarray(alphas), beta=np.asarray(betas), m=m, Q=Q,
                      full_steps=full_steps, omega_max=omega_max)
