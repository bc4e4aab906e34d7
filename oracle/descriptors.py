"""SLQ estimates of the NetLSD heat / wave traces and of the VNGE.

Test infrastructure (see package header).  Functions of the Ritz values:

* heat trace, Eq. heat-trace (Sec. 2.2): h_t = tr exp(-t L) = sum_j exp(-t lambda_j);
* wave trace (NetLSD's second kernel; the paper names NetLSD but prints only
  the heat kernel): w_t = tr exp(-i t L), returned as Re = sum cos(t lambda),
  Im = -sum sin(t lambda);
* VNGE, Definition 1 and Sec. 2.1: H = -sum_i mu_i ln mu_i over the
  eigenvalues mu_i = lambda_i / tr(L) of the density matrix P = L / tr(L),
  natural log, 0 ln 0 = 0; Ritz values theta <= 0 contribute 0.

``slq_runs`` runs Algorithm 1's ``slq`` front half (probes, Lanczos, eigh)
for every probe; the trace functions then apply Eq. slq.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lanczos as _lz
from . import probes as _pr
from . import quadrature as _qd


@dataclass
class ProbeResult:
    alpha: np.ndarray
    beta: np.ndarray
    m: int
    theta: np.ndarray
    tau2: np.ndarray


def slq_runs(lap, s: int, n_v: int, seed: int, graph: int = 0, reorth_passes: int = 1,
             tol: float = _lz.DEFAULT_TOL["fp64"], probes=None,
             partial: bool = False) -> list[ProbeResult]:
    """Lanczos + Gauss rule for probes ``probes`` (default: 0..n_v-1);
    ``partial`` runs Lanczos with partial reorthogonalization instead of
    ``reorth_passes`` Gram-Schmidt passes per step."""
    L = lap.matrix()
    bound = lap.norm_bound()
    out = []
    for p in (range(n_v) if probes is None else probes):
        v = _pr.rademacher(seed, graph, p, lap.old_id)
        if partial:
            run = _lz.lanczos_partial(L, v, s, bound, tol=tol)
        else:
            run = _lz.lanczos(L, v, s, bound, reorth_passes=reorth_passes, tol=tol)
        theta, tau2 = _qd.ritz(run.alpha, run.beta)
        out.append(ProbeResult(run.alpha, run.beta, run.m, theta, tau2))
    return out


def heat_f(t):
    t = np.asarray(t, dtype=np.float64)
    return lambda th: np.exp(-np.multiply.outer(t, th))


def wave_re_f(t):
    t = np.asarray(t, dtype=np.float64)
    return lambda th: np.cos(np.multiply.outer(t, th))


def wave_im_f(t):
    t = np.asarray(t, dtype=np.float64)
    return lambda th: -np.sin(np.multiply.outer(t, th))


def vnge_f(c: float):
    def f(th):
        th = np.asarray(th, dtype=np.float64)
        x = th / c
        out = np.zeros_like(x)
        pos = x > 0
        out[pos] = -x[pos] * np.log(x[pos])
        return out
    return f


def per_probe(runs: list[ProbeResult], f) -> np.ndarray:
    """[n_v, ...] array of sum_k tau_k^2 f(theta_k) for every probe."""
    return np.stack([_qd.quadratic_form(r.theta, r.tau2, f) for r in runs])


def heat_trace(runs, n: int, t):
    return _qd.hutchinson(per_probe(runs, heat_f(t)), n)


def wave_trace(runs, n: int, t):
    re = _qd.hutchinson(per_probe(runs, wave_re_f(t)), n)
    im = _qd.hutchinson(per_probe(runs, wave_im_f(t)), n)
    return re, im


def vnge(runs, n: int, c: float):
    mean, se = _qd.hutchinson(per_probe(runs, vnge_f(c)), n)
    return float(mean), float(se)
