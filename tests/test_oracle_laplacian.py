"""Pins of the oracle's Laplacian builder (Sec. 2) against closed forms and
invariants that hold independently of the builder's code."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import synth
from oracle import exact
from oracle.laplacian import COMBINATORIAL, NORMALIZED, build_laplacian

TOL = 1e-12


def spec(g, kind, **kw):
    s, d, n = g
    return np.sort(exact.spectrum(build_laplacian(s, d, n, kind=kind, **kw)))


# closed-form spectra (Chung, Spectral Graph Theory, Ch. 1; Brouwer-Haemers Ch. 1)
@pytest.mark.parametrize("n", [2, 3, 7])
def test_complete_graph(n):
    assert np.allclose(spec(synth.complete(n), NORMALIZED),
                       [0.0] + [n / (n - 1)] * (n - 1), atol=TOL)
    assert np.allclose(spec(synth.complete(n), COMBINATORIAL), [0.0] + [n] * (n - 1), atol=1e-11)


@pytest.mark.parametrize("n", [3, 4, 9])
def test_cycle(n):
    k = np.arange(n)
    assert np.allclose(spec(synth.cycle(n), NORMALIZED), np.sort(1 - np.cos(2 * np.pi * k / n)), atol=TOL)
    assert np.allclose(spec(synth.cycle(n), COMBINATORIAL), np.sort(2 - 2 * np.cos(2 * np.pi * k / n)), atol=1e-11)


@pytest.mark.parametrize("n", [2, 5, 8])
def test_path(n):
    k = np.arange(n)
    assert np.allclose(spec(synth.path(n), NORMALIZED), np.sort(1 - np.cos(np.pi * k / (n - 1))), atol=TOL)
    assert np.allclose(spec(synth.path(n), COMBINATORIAL), np.sort(2 - 2 * np.cos(np.pi * k / n)), atol=1e-11)


@pytest.mark.parametrize("n", [3, 6, 11])
def test_star(n):
    assert np.allclose(spec(synth.star(n), NORMALIZED), [0.0] + [1.0] * (n - 2) + [2.0], atol=TOL)
    assert np.allclose(spec(synth.star(n), COMBINATORIAL), [0.0] + [1.0] * (n - 2) + [float(n)], atol=1e-11)


@pytest.mark.parametrize("a,b", [(2, 3), (4, 4), (1, 5)])
def test_complete_bipartite(a, b):
    g = synth.complete_bipartite(a, b)
    assert np.allclose(spec(g, NORMALIZED), [0.0] + [1.0] * (a + b - 2) + [2.0], atol=TOL)
    want = np.sort([0.0] + [a] * (b - 1) + [b] * (a - 1) + [a + b])
    assert np.allclose(spec(g, COMBINATORIAL), want, atol=1e-11)


def _random_graph_with_components():
    g1 = synth.erdos_renyi(40, 0.15, seed=4)
    g2 = synth.cycle(7)
    g3 = synth.barabasi_albert(30, 2, seed=5)
    return synth.disjoint_union(g1, g2, g3, extra_isolated=3)


def test_invariants_random_graph():
    s, d, n = _random_graph_with_components()
    A = sp.coo_matrix((np.ones(s.size), (s, d)), shape=(n, n))
    ncomp, _ = connected_components(A + A.T, directed=False)
    deg = np.bincount(np.concatenate([s, d]), minlength=n)
    n_nonisolated = int(np.count_nonzero(deg))
    for kind in (NORMALIZED, COMBINATORIAL):
        lap = build_laplacian(s, d, n, kind=kind)
        lam = exact.spectrum(lap)
        bound = lap.norm_bound()
        assert lam.min() > -1e-12 and lam.max() < bound + 1e-12
        # multiplicity of 0 = number of connected components (isolated nodes count)
        assert np.count_nonzero(np.abs(lam) < 1e-9) == ncomp
        M = lap.dense()
        assert np.array_equal(M, M.T)
    lap = build_laplacian(s, d, n, kind=NORMALIZED)
    assert lap.trace == n_nonisolated
    assert np.isclose(np.trace(lap.dense()), n_nonisolated)
    # D^{1/2} 1 spans the null space of the normalized Laplacian on every component
    sq = np.sqrt(deg.astype(float))
    assert np.max(np.abs(lap.dense() @ sq)) < 1e-12
    # tr(L^2) = sum_ij L_ij^2 (Eq. vnge-taylor text)
    M = lap.dense()
    assert np.isclose(np.trace(M @ M), np.sum(M * M))
    lapc = build_laplacian(s, d, n, kind=COMBINATORIAL)
    assert np.max(np.abs(lapc.dense() @ np.ones(n))) == 0.0
    assert lapc.trace == 2 * len(set(zip(np.minimum(s, d), np.maximum(s, d))))


def test_csr_is_canonical():
    s, d, n = _random_graph_with_components()
    lap = build_laplacian(s, d, n)
    for i in range(lap.n):
        row = lap.colidx[lap.rowptr[i]:lap.rowptr[i + 1]]
        assert np.all(np.diff(row) > 0)       # sorted, no duplicates
        assert not np.any(row == i)           # no self-loops


def test_cleaning_loops_duplicates_orientation():
    s, d, n = synth.barabasi_albert(50, 3, seed=1)
    clean = build_laplacian(s, d, n)
    # add self-loops, reversed duplicates and exact duplicates
    s2 = np.concatenate([s, d[:20], s[:10], np.arange(5)]).astype(np.int32)
    d2 = np.concatenate([d, s[:20], d[:10], np.arange(5)]).astype(np.int32)
    dirty = build_laplacian(s2, d2, n)
    assert np.array_equal(clean.rowptr, dirty.rowptr)
    assert np.array_equal(clean.colidx, dirty.colidx)
    assert np.array_equal(clean.vals, dirty.vals)


def test_drop_isolated_relabels_in_order():
    s, d, n = _random_graph_with_components()
    # move the isolated nodes into the middle of the id range
    perm = np.random.default_rng(0).permutation(n)
    s, d = perm[s].astype(np.int32), perm[d].astype(np.int32)
    full = build_laplacian(s, d, n)
    drop = build_laplacian(s, d, n, drop_isolated=True)
    deg = np.bincount(np.concatenate([s, d]), minlength=n)
    assert np.array_equal(drop.old_id, np.flatnonzero(deg))
    assert drop.n == n - 3
    lam_full = np.sort(exact.spectrum(full))
    lam_drop = np.sort(exact.spectrum(drop))
    assert np.allclose(lam_full[3:], lam_drop, atol=1e-12)
    # the kept sub-matrix is unchanged
    keep = drop.old_id
    assert np.array_equal(full.dense()[np.ix_(keep, keep)], drop.dense())


def test_weights_and_duplicate_merge():
    # weighted path 0-1-2 with weights 2 and 3; a duplicate 1-0 edge of weight 0.5
    s = np.array([0, 1, 1], np.int32)
    d = np.array([1, 2, 0], np.int32)
    w = np.array([2.0, 3.0, 0.5])
    lap = build_laplacian(s, d, 3, weights=w, kind=COMBINATORIAL)
    assert np.array_equal(lap.dense(), np.array([[2., -2, 0], [-2, 5, -3], [0, -3, 3]]))
    lapn = build_laplacian(s, d, 3, weights=w, kind=NORMALIZED)
    lam = np.sort(exact.spectrum(lapn))
    assert abs(lam[0]) < 1e-12 and lam[-1] <= 2 + 1e-12
    # weighted D^{1/2} is the null vector
    assert np.max(np.abs(lapn.dense() @ np.sqrt([2.0, 5.0, 3.0]))) < 1e-12


@pytest.mark.parametrize("bad", [(-1, 0), (0, 5)])
def test_invalid_ids(bad):
    with pytest.raises(ValueError):
        build_laplacian(np.array([bad[0]], np.int32), np.array([bad[1]], np.int32), 5)


def test_empty_graph():
    lap = build_laplacian(np.zeros(0, np.int32), np.zeros(0, np.int32), 4)
    assert lap.n == 4 and lap.nnz == 0 and lap.trace == 0
    lap = build_laplacian(np.zeros(0, np.int32), np.zeros(0, np.int32), 4, drop_isolated=True)
    assert lap.n == 0
