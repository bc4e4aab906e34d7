"""Input generators: determinism, sizes and the structural properties the
workloads ask for (unique non-loop pairs, degree skew, block structure)."""
import numpy as np
import pytest

import synth


def _pairs(s, d):
    return set(zip(np.minimum(s, d).tolist(), np.maximum(s, d).tolist()))


def test_t_grid():
    t = synth.t_grid()
    assert t.size == 256 and t[0] == 1e-2 and t[-1] == 1e2
    assert np.all(np.diff(np.log10(t)) > 0)


def test_barabasi_albert():
    s, d, n = synth.barabasi_albert(500, 4, seed=0)
    assert n == 500 and s.size == 4 + 4 * (500 - 5)
    assert len(_pairs(s, d)) == s.size and not np.any(s == d)
    s2, d2, _ = synth.barabasi_albert(500, 4, seed=0)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    deg = np.bincount(np.concatenate([s, d]))
    assert deg.max() > 5 * np.median(deg)            # preferential attachment skew


def test_rmat_unique_and_skewed():
    s, d, n = synth.rmat(12, 16 << 12, seed=1)
    assert n == 4096 and s.size == 16 << 12
    assert not np.any(s == d)
    assert len(_pairs(s, d)) == s.size
    s2, d2, _ = synth.rmat(12, 16 << 12, seed=1)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    deg = np.bincount(np.concatenate([s, d]), minlength=n)
    assert deg[0] == deg.max()                        # a=0.57: node 0 is the hub
    assert np.count_nonzero(deg == 0) > 0


def test_sbm_batch_shapes():
    gs = synth.sbm_batch(6, seed=3)
    for s, d, n in gs:
        assert 10 <= n <= 5000
        assert len(_pairs(s, d)) == s.size and not np.any(s == d)
        assert s.max(initial=0) < n and d.max(initial=0) < n


def test_rewire_keeps_edge_count():
    s, d, n = synth.barabasi_albert(300, 3, seed=2)
    s2, d2, n2 = synth.rewire(s, d, n, frac=0.01, seed=5)
    a, b = _pairs(s, d), _pairs(s2, d2)
    assert n2 == n and len(b) == len(a)
    k = int(np.ceil(0.01 * len(a)))
    assert len(a - b) == k and len(b - a) == k
    assert not np.any(s2 == d2)


def test_rmat_torch_unique_and_skewed():
    torch = pytest.importorskip("torch")
    s, d, n = synth.rmat_torch(12, 16 << 12, seed=3, device="cpu")
    s, d = s.numpy(), d.numpy()
    assert n == 4096 and s.size == 16 << 12 and s.dtype == np.int32
    assert len(_pairs(s, d)) == s.size and not np.any(s == d)
    deg = np.bincount(np.concatenate([s, d]), minlength=n)
    assert deg.max() > 20 * np.median(deg[deg > 0])     # R-MAT's heavy tail
    s2, d2, _ = synth.rmat_torch(12, 16 << 12, seed=3, device="cpu")
    assert np.array_equal(s, s2.numpy()) and np.array_equal(d, d2.numpy())


def test_rmat_torch_node_restriction_and_rewire_torch():
    """The graph-pair workload's generators, on torch's CPU device here
    (the bench draws them on the GPU): R-MAT on a node count that is not a
    power of two, then a 0.1% rewire that keeps the node set."""
    torch = pytest.importorskip("torch")
    n_i = round(2 ** (10 + 4 * 5 / 63))       # 1268 nodes, scale 11
    s, d, n = synth.rmat_torch(11, 16 * n_i, seed=100, device="cpu", n_nodes=n_i)
    assert n == n_i and s.numel() == 16 * n_i
    s, d = s.numpy(), d.numpy()
    assert s.max() < n_i and d.max() < n_i and not np.any(s == d)
    pairs = _pairs(s, d)
    assert len(pairs) == s.size
    s2, d2, _ = synth.rmat_torch(11, 16 * n_i, seed=100, device="cpu", n_nodes=n_i)
    assert np.array_equal(s, s2.numpy())
    r_s, r_d, rn = synth.rewire_torch(torch.as_tensor(s), torch.as_tensor(d), n_i, frac=1e-3, seed=3)
    new = _pairs(r_s.numpy(), r_d.numpy())
    k = int(np.ceil(1e-3 * len(pairs)))
    assert rn == n_i and len(new) == len(pairs)
    assert len(pairs - new) == k and len(new - pairs) == k
    assert not np.any(r_s.numpy() == r_d.numpy()) and r_s.max() < n_i and r_d.max() < n_i
