"""Pins of the oracle's comparators (Sec. 2.3): the Taylor heat trace of Eq.
hks-taylor, the quadratic VNGE approximation Q, FINGER-Hbar and FINGER-Hhat,
against closed forms written out here, the Taylor remainder bound, the
inequality -x ln x >= x (1 - x) that makes Q a lower bound of the VNGE, and
planted mistakes; and the Erdos-Renyi accuracy comparison of Fig. 4 / Sec. 4.1
(SLQ against the Taylor expansion, relative l2 error of the heat descriptor)
at sizes the oracle finishes in seconds."""
import math

import numpy as np
import pytest

import synth
from oracle import comparators as cmp
from oracle import descriptors, exact
from oracle.laplacian import COMBINATORIAL, NORMALIZED, build_laplacian


def pin_complete_graph():
    n = 11
    for kind in (NORMALIZED, COMBINATORIAL):
        lap = build_laplacian(*synth.complete(n), kind=kind)
        q = 1.0 - 1.0 / (n - 1)   # both Laplacians: tr L^2 / tr L^2 = 1 / (n - 1)
        assert math.isclose(cmp.vnge_quadratic(lap), q, rel_tol=1e-13)
        lam_max = n / (n - 1) if kind == NORMALIZED else float(n)
        assert math.isclose(cmp.finger_hat(lap, lam_max), q * math.log(n - 1), rel_tol=1e-13)
        bar = -q * math.log(2.0 / n) if kind == NORMALIZED else q * math.log(n / 2.0)
        assert math.isclose(cmp.finger_bar(lap), bar, rel_tol=1e-13)
    lap = build_laplacian(*synth.complete(n))
    t = np.array([0.01, 0.5, 3.0])
    np.testing.assert_allclose(cmp.taylor_heat(lap, t),
                               n - t * n + 0.5 * t * t * (n + n / (n - 1)), rtol=1e-14)


def pin_star_combinatorial():
    """Star S_n, L = D - A: eigenvalues {0, 1^(n-2), n}, tr L = 2(n-1),
    tr L^2 = (n-1)^2 + (n-1) + 2(n-1) = (n-1)(n+2)."""
    n = 9
    lap = build_laplacian(*synth.star(n), kind=COMBINATORIAL)
    q = 1.0 - (n - 1) * (n + 2) / (4.0 * (n - 1) ** 2)
    assert math.isclose(cmp.vnge_quadratic(lap), q, rel_tol=1e-13)
    assert math.isclose(cmp.finger_hat(lap, float(n)), -q * math.log(n / (2.0 * (n - 1))), rel_tol=1e-13)
    assert math.isclose(cmp.finger_bar(lap), -q * math.log(2.0 * (n - 1) / (2.0 * (n - 1))) + 0.0,
                        abs_tol=1e-15)  # 2 max d = tr L: the bound of mu_max is 1


def pin_bounds_and_remainder():
    """Q <= H (since -ln x >= 1 - x), Hbar <= Hhat with the exact lambda_max
    (the Gershgorin bound is >= lambda_max), and the Taylor remainder of the
    heat trace <= t^3/6 sum lambda^3."""
    for (s, d, n) in (synth.barabasi_albert(120, 3, seed=1), synth.erdos_renyi(150, 0.05, seed=3),
                      synth.cycle(40)):
        for kind in (NORMALIZED, COMBINATORIAL):
            lap = build_laplacian(s, d, n, kind=kind, drop_isolated=True)
            lam = exact.spectrum(lap)
            h = exact.vnge(lam, lap.trace)
            q = cmp.vnge_quadratic(lap)
            assert 0.0 < q <= h + 1e-12
            assert cmp.finger_bar(lap) <= cmp.finger_hat(lap, lam.max()) + 1e-12
            for tv in (1e-3, 1e-2):
                r = abs(exact.heat_trace(lam, np.array([tv]))[0] - cmp.taylor_heat(lap, np.array([tv]))[0])
                assert r <= tv ** 3 / 6 * np.sum(lam ** 3) * 1.0001 + 1e-12


PINS = [pin_complete_graph, pin_star_combinatorial, pin_bounds_and_remainder]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_comparator_pin(pin):
    pin()


@pytest.mark.parametrize("slip", ["q_printed_taylor", "bar_trace_squared", "taylor_plus_t"])
def test_planted_comparator_mistakes_are_caught(monkeypatch, slip):
    if slip == "q_printed_taylor":   # Eq. vnge-taylor taken literally
        monkeypatch.setattr(cmp, "vnge_quadratic",
                            lambda lap: 1.0 - (lap.trace + 2 * cmp._var.frobenius_sq(lap)) / lap.trace ** 2)
    elif slip == "bar_trace_squared":  # the printed tr(L)^2 under the bound
        monkeypatch.setattr(cmp, "finger_bar",
                            lambda lap: -cmp.vnge_quadratic(lap) * math.log(lap.norm_bound() / lap.trace ** 2))
    else:
        monkeypatch.setattr(cmp, "taylor_heat",
                            lambda lap, t: lap.n + np.asarray(t) * lap.trace
                            + 0.5 * np.asarray(t) ** 2 * cmp._var.frobenius_sq(lap))
    caught = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught >= 1


def test_erdos_renyi_sweep_slq_beats_taylor():
    """Fig. 4's setup at oracle sizes: ER graphs of one size with growing
    density, and of growing size at average degree 10.  The SLQ heat
    descriptor (s = 10, nv = 60) stays within a few 1e-3 of the exact one in
    relative l2 over the t grid, at every size and density, while the Taylor
    expansion, exact only for small t, is off by orders of magnitude more."""
    t = synth.t_grid(64)
    cases = [(300, p) for p in (0.02, 0.05, 0.1, 0.2)] + [(n, 20.0 / n) for n in (100, 200, 400)]
    for i, (n, p) in enumerate(cases):
        s, d, nn = synth.erdos_renyi(n, p, seed=10 + i)
        lap = build_laplacian(s, d, nn, drop_isolated=True)
        ex = exact.heat_trace(exact.spectrum(lap), t)
        runs = descriptors.slq_runs(lap, 10, 60, seed=i)
        h, _ = descriptors.heat_trace(runs, lap.n, t)
        e_slq = cmp.relative_l2(h, ex)
        e_tay = cmp.relative_l2(cmp.taylor_heat(lap, t), ex)
        assert e_slq < 2e-2, (n, p, e_slq)
        assert e_tay > 100 * e_slq, (n, p, e_tay, e_slq)
