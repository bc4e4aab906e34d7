"""Pins of the polynomial control variate (oracle/variance.py).

tr L^2 against closed forms and a dense sum; Chebyshev interpolation and the
control-variate estimate exact for polynomial f (where both the estimate and
its standard error are fixed by the mathematics: the residual f - p is zero);
unbiasedness against the exact spectrum and a smaller standard error than the
plain estimate on the same probes."""
import numpy as np
import pytest

import synth
from oracle import descriptors as od
from oracle import exact as ox
from oracle import variance as ov
from oracle.laplacian import COMBINATORIAL, NORMALIZED, build_laplacian


@pytest.mark.parametrize("n", [5, 12])
def test_frobenius_closed_forms(n):
    kn = build_laplacian(*synth.complete(n))
    assert ov.frobenius_sq(kn) == pytest.approx(n + n / (n - 1), rel=1e-14)
    cn = build_laplacian(*synth.cycle(n))
    assert ov.frobenius_sq(cn) == pytest.approx(1.5 * n, rel=1e-14)
    st = build_laplacian(*synth.star(n))          # n nodes: a center and n - 1 leaves
    assert ov.frobenius_sq(st) == pytest.approx(n + 2.0, rel=1e-14)
    kc = build_laplacian(*synth.complete(n), kind=COMBINATORIAL)
    assert ov.frobenius_sq(kc) == pytest.approx(n * n * (n - 1), rel=1e-14)


def test_frobenius_dense_weighted():
    s, d, n = synth.barabasi_albert(60, 3, seed=2)
    w = np.random.default_rng(1).uniform(0.5, 2.0, s.size)
    for kind in (NORMALIZED, COMBINATORIAL):
        lap = build_laplacian(s, d, n, weights=w, kind=kind)
        dense = lap.dense()
        assert ov.frobenius_sq(lap) == pytest.approx(float(np.sum(dense * dense)), rel=1e-13)
        # tr L^2 is also the sum of the squared eigenvalues
        lam = ox.spectrum(lap)
        assert ov.frobenius_sq(lap) == pytest.approx(float(np.sum(lam * lam)), rel=1e-11)


def test_chebyshev_reproduces_polynomials():
    c1 = ov.chebyshev_coefficients(lambda x: 3.0 - 2.0 * x, 1, 2.0)
    np.testing.assert_allclose(c1, [3.0, -2.0], atol=1e-14)
    c2 = ov.chebyshev_coefficients(lambda x: 1.0 + x - 0.5 * x * x, 2, 7.0)
    np.testing.assert_allclose(c2, [1.0, 1.0, -0.5], atol=1e-13)


@pytest.mark.parametrize("kind", [NORMALIZED, COMBINATORIAL])
def test_cv_exact_for_polynomial_f(kind):
    s, d, n = synth.barabasi_albert(150, 3, seed=4)
    lap = build_laplacian(s, d, n, kind=kind)
    runs = od.slq_runs(lap, 8, 6, seed=3)
    tr_l, tr_l2 = lap.trace, ov.frobenius_sq(lap)
    bound = lap.norm_bound()
    # f of degree 2 with degree-2 control variate: the estimate is exact
    f = lambda x: 0.5 - 0.25 * x + 0.125 * x * x  # noqa: E731
    est, se = ov.trace_cv(runs, lap.n, f, 2, bound, tr_l, tr_l2)
    want = 0.5 * lap.n - 0.25 * tr_l + 0.125 * tr_l2
    assert est == pytest.approx(want, rel=1e-12)
    assert se < 1e-9 * abs(want)
    # degree 1 on a linear f
    est1, se1 = ov.trace_cv(runs, lap.n, lambda x: 2.0 + 3.0 * x, 1, bound, tr_l, tr_l2)
    assert est1 == pytest.approx(2.0 * lap.n + 3.0 * tr_l, rel=1e-12)
    assert se1 < 1e-9 * abs(est1)


def test_cv_unbiased_and_reduces_variance():
    s, d, n = synth.barabasi_albert(300, 3, seed=9)
    lap = build_laplacian(s, d, n)
    lam = ox.spectrum(lap)
    runs = od.slq_runs(lap, 15, 40, seed=7)
    tr_l, tr_l2 = lap.trace, ov.frobenius_sq(lap)
    t = np.array([0.1, 1.0, 5.0])
    exact = ox.heat_trace(lam, t)
    plain, plain_se = od.heat_trace(runs, lap.n, t)
    for degree in (1, 2):
        cv, cv_se = ov.heat_trace_cv(runs, lap.n, t, degree, lap.norm_bound(), tr_l, tr_l2)
        assert np.all(np.abs(cv - exact) <= 3 * cv_se + 1e-9 * exact), degree
        assert np.all(cv_se[:2] < 0.5 * plain_se[:2]), (degree, cv_se, plain_se)
