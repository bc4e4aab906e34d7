"""Pins of the oracle's wave trace tr exp(-i t L), returned as Re = sum cos(t lambda)
and Im = -sum sin(t lambda), against mathematics the oracle does not restate.

The paper names NetLSD's descriptors but prints only the heat kernel (Sec. 2.2);
the wave kernel is NetLSD's second one.  The oracle evaluates it through
``descriptors.wave_re_f`` / ``wave_im_f``, both in the exact-spectrum route
(``exact.wave_trace``) and in the SLQ route (``descriptors.wave_trace``).  These
pins reach the same quantities without those two functions:

* closed forms of the spectra of K_n, the star S_n and the cycle C_n, with the
  trigonometric sums written out here;
* the matrix exponential exp(-i t L) from scipy's Pade-based ``expm`` (no
  eigendecomposition, no cos/sin of eigenvalues): its trace, and q^T exp(-i t L) q
  per probe against the probe's Gauss rule, which is exact up to the Taylor
  remainder of degree 2m;
* the small-t expansion tr exp(-i t L) = n - t^2/2 tr L^2 + ... - i (t tr L -
  t^3/6 tr L^3 + ...), with the remainders bounded by the next term;
* the per-probe breakdown identity on K_n (two distinct eigenvalues).

A planted-mistake test swaps in the plausible slips (+sin for Im, cos(t theta / 2)
for Re, sin for cos, a dropped minus on t) and checks that these pins catch
each of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import descriptors, exact, probes
from oracle.laplacian import COMBINATORIAL, NORMALIZED, build_laplacian

T_GRID = np.array([0.03, 0.4, 1.0, 2.5, 7.0, 31.0])


def _oracle_exact(lap, t):
    return exact.wave_trace(exact.spectrum(lap), t)


# ---------------------------------------------------------------- the pins
def pin_closed_forms():
    """K_n, S_n and C_n (normalized and combinatorial) from their printed spectra."""
    t = T_GRID
    n = 9
    # K_n normalized: {0, n/(n-1) with multiplicity n-1}
    lam = n / (n - 1)
    re, im = _oracle_exact(build_laplacian(*synth.complete(n)), t)
    np.testing.assert_allclose(re, 1 + (n - 1) * np.cos(t * lam), rtol=0, atol=1e-11)
    np.testing.assert_allclose(im, -(n - 1) * np.sin(t * lam), rtol=0, atol=1e-11)
    # K_n combinatorial: {0, n with multiplicity n-1}
    re, im = _oracle_exact(build_laplacian(*synth.complete(n), kind=COMBINATORIAL), t)
    np.testing.assert_allclose(re, 1 + (n - 1) * np.cos(t * n), rtol=0, atol=1e-10)
    np.testing.assert_allclose(im, -(n - 1) * np.sin(t * n), rtol=0, atol=1e-10)
    # star S_n normalized: {0, 1 with multiplicity n-2, 2}
    re, im = _oracle_exact(build_laplacian(*synth.star(n)), t)
    np.testing.assert_allclose(re, 1 + (n - 2) * np.cos(t) + np.cos(2 * t), rtol=0, atol=1e-11)
    np.testing.assert_allclose(im, -(n - 2) * np.sin(t) - np.sin(2 * t), rtol=0, atol=1e-11)
    # cycle C_n normalized: {1 - cos(2 pi k / n)}, k = 0..n-1
    c = 11
    re, im = _oracle_exact(build_laplacian(*synth.cycle(c)), t)
    want_re = np.zeros_like(t)
    want_im = np.zeros_like(t)
    for k in range(c):
        mu = 1.0 - math.cos(2 * math.pi * k / c)
        want_re += np.cos(t * mu)
        want_im -= np.sin(t * mu)
    np.testing.assert_allclose(re, want_re, rtol=0, atol=1e-11)
    np.testing.assert_allclose(im, want_im, rtol=0, atol=1e-11)


def pin_matrix_exponential():
    """tr exp(-i t L) through scipy's Pade matrix exponential (both Laplacians)."""
    s, d, n = synth.barabasi_albert(70, 3, seed=4)
    for kind in (NORMALIZED, COMBINATORIAL):
        lap = build_laplacian(s, d, n, kind=kind)
        M = lap.dense()
        t = T_GRID if kind == NORMALIZED else T_GRID[:4] / 10
        re, im = _oracle_exact(lap, t)
        for i, tv in enumerate(t):
            tr = np.trace(scipy.linalg.expm(-1j * tv * M))
            assert abs(re[i] - tr.real) <= 1e-9 * n, (kind, tv, re[i], tr.real)
            assert abs(im[i] - tr.imag) <= 1e-9 * n, (kind, tv, im[i], tr.imag)


def pin_probe_quadrature_vs_expm():
    """Per probe, the Gauss rule of the oracle's Lanczos run integrates
    exp(-i t x) up to its Taylor remainder (t ||L||)^(2m) / (2m)!; the
    reference value q^T exp(-i t L) q comes from scipy's expm."""
    s, d, n = synth.barabasi_albert(120, 3, seed=6)
    lap = build_laplacian(s, d, n)
    M = lap.dense()
    steps = 8
    runs = descriptors.slq_runs(lap, s=steps, n_v=3, seed=13)
    t = np.array([0.1, 0.3, 0.6])
    re_pp = descriptors.per_probe(runs, descriptors.wave_re_f(t))
    im_pp = descriptors.per_probe(runs, descriptors.wave_im_f(t))
    for p in range(3):
        q = probes.rademacher(13, 0, p, lap.old_id)
        q = q / np.linalg.norm(q)
        for i, tv in enumerate(t):
            want = q @ scipy.linalg.expm(-1j * tv * M) @ q
            rem = (tv * 2.0) ** (2 * steps) / math.factorial(2 * steps)
            assert abs(re_pp[p, i] - want.real) <= rem + 1e-13, (p, tv)
            assert abs(im_pp[p, i] - want.imag) <= rem + 1e-13, (p, tv)
    # the Hutchinson mean of the SLQ route is n' times the probe average
    (wr, _), (wi, _) = descriptors.wave_trace(runs, lap.n, t)
    np.testing.assert_allclose(wr, lap.n * re_pp.mean(0), rtol=1e-14)
    np.testing.assert_allclose(wi, lap.n * im_pp.mean(0), rtol=1e-14)


def pin_small_t():
    """Re = n - t^2/2 tr L^2 + R, |R| <= t^4/24 sum lambda^4;
    Im = -t tr L + t^3/6 tr L^3 + R', |R'| <= t^5/120 sum lambda^5;
    the traces of powers from dense matrix products."""
    s, d, n = synth.barabasi_albert(150, 3, seed=8)
    lap = build_laplacian(s, d, n)
    M = lap.dense()
    lam = exact.spectrum(lap)
    M2 = M @ M
    tr1, tr2, tr3 = np.trace(M), np.trace(M2), np.trace(M2 @ M)
    for tv in (1e-3, 1e-2, 5e-2):
        re, im = exact.wave_trace(lam, np.array([tv]))
        r_re = abs(re[0] - (lap.n - tv * tv / 2 * tr2))
        r_im = abs(im[0] - (-tv * tr1 + tv ** 3 / 6 * tr3))
        assert r_re <= tv ** 4 / 24 * np.sum(lam ** 4) * 1.0001 + 1e-12 * lap.n, (tv, r_re)
        assert r_im <= tv ** 5 / 120 * np.sum(lam ** 5) * 1.0001 + 1e-12 * lap.n, (tv, r_im)
        # and the first dropped term is really there (the expansion is not trivially met)
        assert abs(re[0] - lap.n) >= tv * tv / 2 * tr2 * 0.99
        assert abs(im[0]) >= tv * tr1 * 0.99


def pin_complete_graph_per_probe():
    """K_n, normalized: the Krylov space of q closes after 2 steps, so per
    probe the rule is exact: with S = sum v_i and a = S^2 / n^2,
    q^T cos(tL) q = a + (1 - a) cos(t n/(n-1)), -q^T sin(tL) q = -(1 - a) sin(t n/(n-1))."""
    n = 13
    lap = build_laplacian(*synth.complete(n))
    runs = descriptors.slq_runs(lap, s=6, n_v=5, seed=17)
    t = T_GRID
    re_pp = descriptors.per_probe(runs, descriptors.wave_re_f(t))
    im_pp = descriptors.per_probe(runs, descriptors.wave_im_f(t))
    lam = n / (n - 1)
    for p in range(5):
        S = probes.rademacher(17, 0, p, lap.old_id).sum()
        a = S * S / n ** 2
        np.testing.assert_allclose(re_pp[p], a + (1 - a) * np.cos(t * lam), rtol=0, atol=1e-13)
        np.testing.assert_allclose(im_pp[p], -(1 - a) * np.sin(t * lam), rtol=0, atol=1e-13)


PINS = [pin_closed_forms, pin_matrix_exponential, pin_probe_quadrature_vs_expm, pin_small_t,
        pin_complete_graph_per_probe]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_wave_pin(pin):
    pin()


# ------------------------------------------------------- planted mistakes
def _re_half(t):
    t = np.asarray(t, dtype=np.float64)
    return lambda th: np.cos(np.multiply.outer(t, th) / 2)


def _im_plus(t):
    t = np.asarray(t, dtype=np.float64)
    return lambda th: np.sin(np.multiply.outer(t, th))


def _re_sin(t):
    t = np.asarray(t, dtype=np.float64)
    return lambda th: np.sin(np.multiply.outer(t, th))


def _im_neg_t(t):  # -sin(-t theta): the sign of t dropped in the argument
    t = np.asarray(t, dtype=np.float64)
    return lambda th: -np.sin(-np.multiply.outer(t, th))


@pytest.mark.parametrize("attr,bad", [("wave_im_f", _im_plus), ("wave_re_f", _re_half),
                                      ("wave_re_f", _re_sin), ("wave_im_f", _im_neg_t)],
                         ids=["im_plus_sin", "re_cos_half", "re_sin", "im_sign_of_t"])
def test_planted_wave_mistakes_are_caught(monkeypatch, attr, bad):
    """Each slip, planted in the oracle on the CPU, breaks at least one pin."""
    monkeypatch.setattr(descriptors, attr, bad)
    caught = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught >= 1, f"no pin caught the planted {attr} mistake"
