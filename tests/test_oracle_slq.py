"""Pins of the oracle's Lanczos, Gauss rule and Hutchinson estimate (Sec. 3.1,
Eq. quadratic, Eq. slq, Algorithm 1) against mathematics the code does not
restate: Gauss-rule moment exactness, T = Q^T L Q, exactness on graphs with
few distinct eigenvalues, the small-t Taylor expansion (Eq. hks-taylor), the
Lanczos error bound (Eq. eps2) and the Monte-Carlo error of Eq. trace."""
import math

import numpy as np
import pytest

import synth
from oracle import descriptors, exact, lanczos, probes, quadrature
from oracle.laplacian import COMBINATORIAL, NORMALIZED, build_laplacian


def _ba(n=300, m=3, seed=2, kind=NORMALIZED):
    s, d, nn = synth.barabasi_albert(n, m, seed)
    return build_laplacian(s, d, nn, kind=kind)


@pytest.mark.parametrize("kind", [NORMALIZED, COMBINATORIAL])
def test_moment_identity(kind):
    """An m-point Gauss rule integrates x^j exactly for j <= 2m-1:
    sum_k tau_k^2 theta_k^j = q0^T L^j q0, the right side by repeated matvec."""
    lap = _ba(kind=kind)
    L = lap.matrix()
    scale = lap.norm_bound()
    for p in range(3):
        v = probes.rademacher(11, 0, p, lap.old_id)
        run = lanczos.lanczos(L, v, 8, lap.norm_bound())
        assert run.m == 8
        theta, tau2 = quadrature.ritz(run.alpha, run.beta)
        q = v / np.linalg.norm(v)
        x = q.copy()
        for j in range(2 * run.m):
            lhs = np.sum(tau2 * theta ** j)
            rhs = q @ x
            assert abs(lhs - rhs) <= 1e-10 * scale ** j, (j, lhs, rhs)
            x = L @ x


def test_basis_orthonormal_and_tridiagonal():
    lap = _ba(n=400)
    L = lap.matrix()
    v = probes.rademacher(3, 0, 0, lap.old_id)
    run = lanczos.lanczos(L, v, 20, lap.norm_bound(), keep_basis=True)
    Q = run.Q
    assert np.max(np.abs(Q.T @ Q - np.eye(run.m))) < 1e-12
    T = np.diag(run.alpha) + np.diag(run.beta, 1) + np.diag(run.beta, -1)
    assert np.max(np.abs(Q.T @ (L @ Q) - T)) < 1e-12
    assert np.all(run.beta > 0)
    # first column is the normalized probe
    assert np.allclose(Q[:, 0], v / math.sqrt(lap.n), atol=0, rtol=0)
    # alpha_0 = v^T L v / n
    assert math.isclose(run.alpha[0], v @ (L @ v) / lap.n, rel_tol=1e-13)


def test_cgs2_matches_cgs_on_well_conditioned_graph():
    lap = _ba(n=400)
    L = lap.matrix()
    v = probes.rademacher(3, 0, 0, lap.old_id)
    r1 = lanczos.lanczos(L, v, 15, 2.0, reorth_passes=1)
    r2 = lanczos.lanczos(L, v, 15, 2.0, reorth_passes=2)
    assert np.allclose(r1.alpha, r2.alpha, rtol=1e-12, atol=1e-13)
    assert np.allclose(r1.beta, r2.beta, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("graph,kind,mmax", [
    (synth.complete(9), NORMALIZED, 2), (synth.complete(9), COMBINATORIAL, 2),
    (synth.star(10), NORMALIZED, 3), (synth.star(10), COMBINATORIAL, 3),
    (synth.complete_bipartite(3, 5), NORMALIZED, 3),
    (synth.complete_bipartite(3, 5), COMBINATORIAL, 4),
])
def test_breakdown_and_exactness(graph, kind, mmax):
    """With k distinct eigenvalues the Krylov space has dimension <= k: Lanczos
    breaks down at m <= k and the Gauss rule is then exact for every f."""
    s, d, n = graph
    lap = build_laplacian(s, d, n, kind=kind)
    runs = descriptors.slq_runs(lap, s=10, n_v=6, seed=1)
    t = np.array([0.05, 0.7, 4.0])
    for p, r in enumerate(runs):
        assert 1 <= r.m <= mmax
        v = probes.rademacher(1, 0, p, lap.old_id)
        want = exact.quadratic_form(lap, v, descriptors.heat_f(t))
        got = quadrature.quadratic_form(r.theta, r.tau2, descriptors.heat_f(t))
        assert np.allclose(got, want, rtol=1e-12, atol=1e-13)


def test_complete_graph_closed_form():
    """K_n, normalized: for unit q = v/sqrt(n) with S = sum v_i the quadratic
    form is (S^2/n^2) f(0) + (1 - S^2/n^2) f(n/(n-1))."""
    n = 11
    lap = build_laplacian(*synth.complete(n))
    runs = descriptors.slq_runs(lap, s=6, n_v=5, seed=4)
    t = 0.9
    for p, r in enumerate(runs):
        S = probes.rademacher(4, 0, p, lap.old_id).sum()
        want = (S * S / n ** 2) * 1.0 + (1 - S * S / n ** 2) * math.exp(-t * n / (n - 1))
        got = float(np.sum(r.tau2 * np.exp(-t * r.theta)))
        assert math.isclose(got, want, rel_tol=1e-13)


def test_weights_sum_to_one_and_h0():
    lap = _ba()
    runs = descriptors.slq_runs(lap, s=10, n_v=8, seed=0)
    for r in runs:
        assert abs(r.tau2.sum() - 1.0) < 1e-13
    h, se = descriptors.heat_trace(runs, lap.n, np.array([0.0]))
    assert abs(h[0] - lap.n) < 1e-10 * lap.n
    assert se[0] < 1e-10 * lap.n


def test_ritz_against_dense_eigh():
    rng = np.random.default_rng(0)
    for m in (1, 2, 3, 7, 20):
        a = rng.uniform(0, 2, m)
        b = rng.uniform(0.01, 1, m - 1)
        th, t2 = quadrature.ritz(a, b)
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        lam, U = np.linalg.eigh(T)
        assert np.allclose(th, lam, atol=1e-13)
        assert np.allclose(t2, U[0] ** 2, atol=1e-13)
    # 2x2 closed form
    a, b, c = 0.3, 1.1, 0.4
    th, t2 = quadrature.ritz(np.array([a, b]), np.array([c]))
    mid, rad = (a + b) / 2, math.hypot((a - b) / 2, c)
    assert np.allclose(th, [mid - rad, mid + rad], atol=1e-15)
    # weight of the lower node: cos^2 of the rotation angle
    assert math.isclose(t2[0], 0.5 * (1 + (b - a) / (2 * rad)), rel_tol=1e-13)


def test_small_t_taylor():
    """Eq. hks-taylor: h_t = n - t tr L + t^2/2 tr L^2 + R, |R| <= t^3/6 sum lambda^3."""
    lap = _ba(n=200)
    lam = exact.spectrum(lap)
    M = lap.dense()
    t = 1e-2
    taylor = lap.n - t * np.trace(M) + t * t / 2 * np.sum(M * M)
    h = exact.heat_trace(lam, np.array([t]))[0]
    assert abs(h - taylor) <= t ** 3 / 6 * np.sum(lam ** 3) * 1.0001
    assert abs(h - taylor) >= t ** 3 / 6 * np.sum(lam ** 3) * np.exp(-2 * t) * 0.9999
    # per probe, the SLQ quadratic form obeys the same expansion in q^T L^j q
    L = lap.matrix()
    runs = descriptors.slq_runs(lap, s=6, n_v=3, seed=2)
    for p, r in enumerate(runs):
        q = probes.rademacher(2, 0, p, lap.old_id)
        q = q / np.linalg.norm(q)
        Lq = L @ q
        tay = 1 - t * (q @ Lq) + t * t / 2 * (Lq @ Lq)
        got = float(np.sum(r.tau2 * np.exp(-t * r.theta)))
        assert abs(got - tay) <= t ** 3 / 6 * 8


def _eps2(s, t):
    if s >= t:
        return 40 / t * math.exp(-0.5 * t) * (0.5 * math.e * t / s) ** s
    if math.sqrt(2 * t) <= s <= t:
        return 20 * math.exp(-s * s / (2.5 * t))
    return math.inf


def test_lanczos_error_bound_eps2():
    """Per-probe quadrature error of exp(-tL) against the exact quadratic form
    stays below the bound of Eq. eps2 (quoted from a cited work; loose)."""
    lap = _ba(n=250)
    s = 8
    runs = descriptors.slq_runs(lap, s=s, n_v=3, seed=5)
    for t in (0.5, 2.0, 5.0, 20.0, 50.0):
        for p, r in enumerate(runs):
            v = probes.rademacher(5, 0, p, lap.old_id)
            want = exact.quadratic_form(lap, v, descriptors.heat_f(np.array([t])))[0]
            got = float(np.sum(r.tau2 * np.exp(-t * r.theta)))
            assert abs(got - want) <= _eps2(s, t) + 1e-14, (t, got, want)


def test_slq_against_exact_spectrum():
    """Eq. trace: the Hutchinson mean is within 3 standard errors of the exact
    trace at a few fixed t (no multiple-comparison sweep) and for VNGE."""
    lap = _ba(n=400, m=4, seed=9)
    lam = exact.spectrum(lap)
    runs = descriptors.slq_runs(lap, s=15, n_v=150, seed=21)
    t = np.array([0.01, 0.1, 1.0, 10.0])
    h, se = descriptors.heat_trace(runs, lap.n, t)
    ex = exact.heat_trace(lam, t)
    assert np.all(np.abs(h - ex) <= 3 * se + 1e-9)
    (wr, wrse), (wi, wise) = descriptors.wave_trace(runs, lap.n, t)
    er, ei = exact.wave_trace(lam, t)
    assert np.all(np.abs(wr - er) <= 3 * wrse + 1e-9)
    assert np.all(np.abs(wi - ei) <= 3 * wise + 1e-9)
    v, vse = descriptors.vnge(runs, lap.n, lap.trace)
    assert abs(v - exact.vnge(lam, lap.trace)) <= 3 * vse
    # relative l2 error of the descriptor (the measure of Sec. 4.1), of the
    # order Sec. 4.4 reports for s = 10
    assert np.linalg.norm(h - ex) / np.linalg.norm(ex) < 1e-3


def test_vnge_closed_forms():
    """VNGE of the normalized Laplacian: K_n -> ln(n-1); star S_n ->
    ((n-2)/n) ln n + (2/n) ln(n/2)."""
    n = 9
    lap = build_laplacian(*synth.complete(n))
    assert math.isclose(exact.vnge(exact.spectrum(lap), lap.trace), math.log(n - 1), rel_tol=1e-12)
    runs = descriptors.slq_runs(lap, s=5, n_v=4, seed=3)
    # exact per probe on K_n (two distinct eigenvalues), and unbiased in mean
    est, se = descriptors.vnge(runs, lap.n, lap.trace)
    assert abs(est - math.log(n - 1)) <= 3 * se + 1e-12
    lap = build_laplacian(*synth.star(n))
    want = (n - 2) / n * math.log(n) + 2 / n * math.log(n / 2)
    assert math.isclose(exact.vnge(exact.spectrum(lap), lap.trace), want, rel_tol=1e-12)


def test_isolated_nodes_kept_count_as_zero_eigenvalues():
    g = synth.disjoint_union(synth.cycle(6), synth.path(5), extra_isolated=4)
    lap = build_laplacian(*g)
    runs = descriptors.slq_runs(lap, s=10, n_v=50, seed=8)
    h, se = descriptors.heat_trace(runs, lap.n, np.array([0.0, 1e4]))
    assert math.isclose(h[0], 15.0, rel_tol=1e-12)
    # at very large t only the zero eigenvalues (6 = 2 components + 4 isolated) survive
    assert abs(h[1] - 6.0) <= 3 * se[1] + 1e-9
