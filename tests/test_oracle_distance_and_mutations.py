"""Distance pins, and checks that the pins above catch plausible mistakes
planted in the oracle (on the CPU): a flipped sign, a dropped scale, a wrong
index, a transposed operand."""
import math
import os

import numpy as np
import pytest

import synth
from oracle import descriptors, distance, exact, lanczos, probes, quadrature
from oracle.laplacian import COMBINATORIAL, build_laplacian


def test_distance_pins():
    assert distance.heat_distance([3.0, 0.0], [0.0, 4.0]) == 5.0
    assert distance.wave_distance([1.0], [0.0], [0.0], [1.0]) == math.sqrt(2.0)
    assert distance.vnge_distance(3.846, 3.154) == pytest.approx(0.692, abs=1e-12)
    rng = np.random.default_rng(1)
    a, b, c = rng.normal(size=(3, 16))
    assert distance.heat_distance(a, a) == 0.0
    assert distance.heat_distance(a, b) == distance.heat_distance(b, a)
    assert distance.heat_distance(a, c) <= distance.heat_distance(a, b) + distance.heat_distance(b, c)


def _karate(golden_dir):
    s, d, n = synth.read_edge_file(os.path.join(golden_dir, "karate_fig1.txt"))
    return build_laplacian(s, d, n, kind=COMBINATORIAL)


def test_planted_vnge_sign_is_caught(golden_dir):
    lap = _karate(golden_dir)
    lam = exact.spectrum(lap)
    x = lam[lam > 0] / lap.trace
    assert round(float(np.sum(x * np.log(x))), 3) != 3.154      # sign flipped
    assert round(float(-np.sum(x * np.log2(x))), 3) != 3.154    # wrong log base


def test_planted_hutchinson_scale_is_caught():
    lap = build_laplacian(*synth.barabasi_albert(100, 2, 0))
    runs = descriptors.slq_runs(lap, s=6, n_v=4, seed=0)
    per = descriptors.per_probe(runs, descriptors.heat_f(np.array([0.0])))
    # Algorithm 1's printed 1/n_v (no n) misses h_0 = n
    assert abs(per.mean() - lap.n) > 1.0
    mean, _ = quadrature.hutchinson(per, lap.n)
    assert abs(mean[0] - lap.n) < 1e-9


def test_planted_weight_index_is_caught():
    """Using the LAST eigenvector row for tau breaks the moment identity."""
    lap = build_laplacian(*synth.barabasi_albert(200, 3, 1))
    L = lap.matrix()
    v = probes.rademacher(2, 0, 0, lap.old_id)
    run = lanczos.lanczos(L, v, 6, 2.0)
    from scipy.linalg import eigh_tridiagonal
    th, U = eigh_tridiagonal(run.alpha, run.beta)
    q = v / np.linalg.norm(v)
    rhs = q @ (L @ q)
    assert abs(np.sum(U[0] ** 2 * th) - rhs) < 1e-12
    assert abs(np.sum(U[-1] ** 2 * th) - rhs) > 1e-6


def test_planted_missing_three_term_is_caught():
    """Dropping the beta_{k-1} q_{k-1} term AND the reorthogonalization breaks
    T = Q^T L Q; the oracle with its steps intact satisfies it."""
    lap = build_laplacian(*synth.barabasi_albert(200, 3, 1))
    L = lap.matrix()
    v = probes.rademacher(2, 0, 0, lap.old_id)
    q0 = v / np.linalg.norm(v)
    w = L @ q0
    a0 = q0 @ w
    w = w - a0 * q0
    b0 = np.linalg.norm(w)
    q1 = w / b0
    w = L @ q1
    a1 = q1 @ w
    w_bad = w - a1 * q1                     # beta_0 q_0 term dropped
    assert abs(q0 @ w_bad) > 1e-3
    run = lanczos.lanczos(L, v, 3, 2.0, keep_basis=True)
    assert abs(run.Q[:, 0] @ run.Q[:, 2]) < 1e-14


def test_planted_transposed_scale_is_caught():
    """A normalized Laplacian built with D^{-1} A (one-sided scaling) is not
    symmetric and fails the D^{1/2} null-vector pin."""
    s, d, n = synth.barabasi_albert(60, 2, 3)
    lap = build_laplacian(s, d, n)
    A = -lap.dense() + np.diag(lap.diag)
    A = np.where(A != 0, 1.0, 0.0)
    deg = A.sum(1)
    wrong = np.eye(n) - A / deg[:, None]
    assert np.max(np.abs(wrong @ np.sqrt(deg))) > 1e-3
    assert np.max(np.abs(lap.dense() @ np.sqrt(deg))) < 1e-12
