"""Pins of the oracle's Lanczos with partial reorthogonalization
(oracle/lanczos.py ``lanczos_partial``; Simon's omega-recurrence, not in the
paper) against what the mathematics fixes independently of its code:

* the basis stays semi-orthogonal, max |Q^T Q - I| well below 1e-6, on runs
  where the plain three-term recurrence loses orthogonality completely;
* the omega estimates track the measured q_{k+1}^T q_j (within three orders
  of magnitude either way);
* it reorthogonalizes few steps, in pairs;
* the Gauss rule is still exact for polynomials of degree <= 2m - 1
  (q0^T L^j q0 by repeated matvec), and the heat / wave / VNGE estimates equal
  those of full reorthogonalization within 1e-10;
* plausible mistakes planted in the omega-recurrence (on the CPU) each break
  one of the pins above."""
import math

import numpy as np
import pytest

import synth
from oracle import descriptors, lanczos, probes, quadrature
from oracle.laplacian import COMBINATORIAL, NORMALIZED, build_laplacian


def _graphs():
    return {
        "ba2000": (synth.barabasi_albert(2000, 4, seed=0), NORMALIZED),
        "rmat12": (synth.rmat(12, 16 << 12, seed=3), NORMALIZED),
    }


def _run(name, s=80, kind=None):
    (src, dst, n), k0 = _graphs()[name]
    lap = build_laplacian(src, dst, n, kind=kind or k0, drop_isolated=True)
    L = lap.matrix()
    v = probes.rademacher(1, 0, 0, lap.old_id)
    return lap, L, v, lanczos.lanczos_partial(L, v, s, lap.norm_bound(), keep_basis=True)


def _orth(Q):
    return float(np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))))


def _estimate_ratios(run):
    """max over steps of estimate / measured (measured floored at 1e-15) and
    min of estimate / measured where the measured level exceeds 1e-12, over
    the steps whose new vector was not reorthogonalized."""
    Q = run.Q
    hi, lo = 0.0, math.inf
    for k in range(1, run.m - 1):
        if k in run.full_steps:
            continue
        meas = float(np.max(np.abs(Q[:, :k].T @ Q[:, k + 1])))
        hi = max(hi, run.omega_max[k] / max(meas, 1e-15))
        if meas > 1e-12:
            lo = min(lo, run.omega_max[k] / meas)
    return hi, lo


def _pins_hold(run, s):
    hi, lo = _estimate_ratios(run)
    return (_orth(run.Q) < 1e-6 and hi < 1e3 and lo > 1e-3
            and len(run.full_steps) <= s // 4)


@pytest.mark.parametrize("name", ["ba2000", "rmat12"])
def test_semi_orthogonal_where_plain_lanczos_is_not(name):
    lap, L, v, run = _run(name)
    assert run.m == 80
    assert _orth(run.Q) < 1e-6
    # the three-term recurrence alone, same start
    q = [v / np.linalg.norm(v)]
    b = 0.0
    for k in range(79):
        w = L @ q[k]
        a = q[k] @ w
        w = w - a * q[k] - (b * q[k - 1] if k > 0 else 0.0)
        b = np.linalg.norm(w)
        q.append(w / b)
    assert _orth(np.column_stack(q)) > 1e-2


@pytest.mark.parametrize("name", ["ba2000", "rmat12"])
def test_omega_estimates_track_measured_orthogonality(name):
    _, _, _, run = _run(name)
    hi, lo = _estimate_ratios(run)
    assert hi < 1e3 and lo > 1e-3, (hi, lo)


@pytest.mark.parametrize("name", ["ba2000", "rmat12"])
def test_reorthogonalizes_few_steps_in_pairs(name):
    _, _, _, run = _run(name)
    f = run.full_steps
    assert 2 <= len(f) <= 80 // 4
    assert len(f) % 2 == 0 and all(f[i + 1] == f[i] + 1 for i in range(0, len(f), 2))


@pytest.mark.parametrize("kind", [NORMALIZED, COMBINATORIAL])
def test_gauss_rule_moments_exact(kind):
    lap, L, v, run = _run("ba2000", s=40, kind=kind)
    assert run.full_steps  # the test covers a run that did reorthogonalize
    theta, tau2 = quadrature.ritz(run.alpha, run.beta)
    scale = lap.norm_bound()
    q = v / np.linalg.norm(v)
    x = q.copy()
    for j in range(2 * run.m):
        assert abs(np.sum(tau2 * theta ** j) - q @ x) <= 1e-10 * scale ** j, j
        x = L @ x


@pytest.mark.parametrize("name", ["ba2000", "rmat12"])
def test_descriptors_equal_full_reorthogonalization(name):
    (src, dst, n), _ = _graphs()[name]
    lap = build_laplacian(src, dst, n, drop_isolated=True)
    t = synth.t_grid(64)
    full = descriptors.slq_runs(lap, 40, 4, seed=7)
    part = descriptors.slq_runs(lap, 40, 4, seed=7, partial=True)
    for f in (descriptors.heat_f(t), descriptors.wave_re_f(t), descriptors.wave_im_f(t)):
        a = np.array([quadrature.quadratic_form(r.theta, r.tau2, f) for r in full])
        b = np.array([quadrature.quadratic_form(r.theta, r.tau2, f) for r in part])
        assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(a))
    va, _ = descriptors.vnge(full, lap.n, lap.trace)
    vb, _ = descriptors.vnge(part, lap.n, lap.trace)
    assert abs(va - vb) <= 1e-10 * abs(va)


def test_fp32_unit_roundoff_reorthogonalizes_more_often():
    """The threshold follows the arithmetic: with eps = 2^-24 the run keeps
    |q_i^T q_j| near 2^-12 instead of 2^-26.5 and needs more full steps."""
    lap, L, v, run64 = _run("rmat12", s=40)
    run32 = lanczos.lanczos_partial(L, v, 40, lap.norm_bound(), eps=2.0 ** -24, keep_basis=True)
    assert len(run32.full_steps) >= len(run64.full_steps)
    assert _orth(run32.Q) < 1e-2


def _drop_previous_row(orig):
    return lambda al, be, cur, prev, beta, eps: orig(al, be, cur, [0.0] * len(prev), beta, eps)


def _flip_alpha(orig):
    def f(al, be, cur, prev, beta, eps):
        a2 = list(al)
        a2[-1] = -a2[-1]
        return orig(a2, be, cur, prev, beta, eps)
    return f


def _no_division(orig):
    def f(al, be, cur, prev, beta, eps):
        out = orig(al, be, cur, prev, beta, eps)
        return [x * beta if i < len(out) - 2 else x for i, x in enumerate(out)]
    return f


def _shifted_index(orig):
    def f(al, be, cur, prev, beta, eps):
        k = len(al) - 1
        return orig(al, be, [cur[max(j - 2, 0)] if j < k else cur[j] for j in range(len(cur))],
                    prev, beta, eps)
    return f


@pytest.mark.parametrize("plant", [_drop_previous_row, _flip_alpha, _no_division, _shifted_index])
def test_planted_omega_mistakes_are_caught(plant, monkeypatch):
    _, _, _, ok = _run("ba2000")
    assert _pins_hold(ok, 80)
    monkeypatch.setattr(lanczos, "_omega_next", plant(lanczos._omega_next))
    _, _, _, bad = _run("ba2000")
    assert not _pins_hold(bad, 80)
