"""Pin: the worked example of Fig. 1 (panel b) prints the VNGE of the two
graphs whose edge lists panel (a) prints: Karate H = 3.154, Dolphins H = 3.846.
Only the combinatorial Laplacian L = D - A scaled by its trace (Sec. 2.1) with
the natural log reproduces both, which fixes the paper's VNGE definition."""
import os

import numpy as np
import pytest

import synth
from oracle import descriptors, exact
from oracle.laplacian import COMBINATORIAL, NORMALIZED, build_laplacian

CASES = [("karate_fig1.txt", 34, 78, 3.154), ("dolphins_fig1.txt", 62, 159, 3.846)]


@pytest.mark.parametrize("fname,n,m,printed", CASES)
def test_fig1_vnge_exact(golden_dir, fname, n, m, printed):
    s, d, nn = synth.read_edge_file(os.path.join(golden_dir, fname))
    assert nn == n and s.size == m
    lap = build_laplacian(s, d, n, kind=COMBINATORIAL)
    h = exact.vnge(exact.spectrum(lap), lap.trace)
    assert round(h, 3) == printed
    # the normalized Laplacian does NOT reproduce the printed value
    lapn = build_laplacian(s, d, n, kind=NORMALIZED)
    assert round(exact.vnge(exact.spectrum(lapn), lapn.trace), 3) != printed


@pytest.mark.parametrize("fname,n,m,printed", CASES)
def test_fig1_vnge_slq(golden_dir, fname, n, m, printed):
    """SLQ estimate of the same VNGE is within 3 standard errors of the exact one."""
    s, d, nn = synth.read_edge_file(os.path.join(golden_dir, fname))
    lap = build_laplacian(s, d, n, kind=COMBINATORIAL)
    runs = descriptors.slq_runs(lap, s=12, n_v=200, seed=7)
    est, se = descriptors.vnge(runs, lap.n, lap.trace)
    h = exact.vnge(exact.spectrum(lap), lap.trace)
    assert abs(est - h) <= 3 * se + 1e-12
    assert abs(est - h) / h < 2e-2
