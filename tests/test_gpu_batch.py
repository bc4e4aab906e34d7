"""Batches of graphs as one block-diagonal Laplacian, through the C ABI.

Every graph g of a batch must give what the oracle gives for that graph on
its own with probe graph field g (FP64: relative 1e-10), and what a
single-graph GPU run with graph_id = g gives."""
import numpy as np
import pytest

import synth
from oracle import descriptors as odesc
from oracle.laplacian import COMBINATORIAL, NORMALIZED, build_laplacian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2003_01282_gb300 import slaq  # noqa: E402
from paper_2003_01282_gb300.build import build  # noqa: E402

RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build()
    slaq.lib()


def mixed_batch():
    return [
        synth.barabasi_albert(300, 3, seed=1),
        synth.sbm([40, 40, 41], 0.3, 0.02, seed=2),
        synth.star(30),
        synth.complete(9),
        synth.cycle(17),
        synth.disjoint_union(synth.path(12), synth.cycle(6), extra_isolated=4),
        synth.path(10),
        synth.rmat(11, 8 << 11, seed=4),
        synth.star(2600),                  # a 2599-entry row: split into chunks
    ]


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("kind,drop", [(NORMALIZED, False), (NORMALIZED, True), (COMBINATORIAL, False)])
def test_batch_matches_oracle_per_graph(kind, drop):
    graphs = mixed_batch()
    nv, s, seed = 6, 10, 5
    k = slaq.NORMALIZED if kind == NORMALIZED else slaq.COMBINATORIAL
    gb = slaq.build_laplacian_batch(graphs, kind=k, flags=slaq.DROP_ISOLATED if drop else 0)
    info = slaq.graph_batch_info(gb)
    assert info["n_graphs"] == len(graphs)
    K = slaq.lanczos(gb, nv, s, seed, precision=slaq.FP64)
    alpha, beta, m = (x.cpu().numpy() for x in slaq.krylov_export(K))
    theta, tau2 = (x.cpu().numpy() for x in slaq.ritz_export(K))
    t = synth.t_grid(64)
    heat = slaq.trace_heat(K, _dev(t, torch.float64))[0].cpu().numpy()
    vnge = slaq.trace_vnge(K)[0].cpu().numpy()
    assert heat.shape == (len(graphs), 64) and vnge.shape == (len(graphs),)
    for g, (src, dst, n) in enumerate(graphs):
        lap = build_laplacian(src, dst, n, kind=kind, drop_isolated=drop)
        assert info["node_off"][g + 1] - info["node_off"][g] == lap.n
        assert info["trace"][g] == lap.trace
        runs = odesc.slq_runs(lap, s, nv, seed, graph=g)
        for p, r in enumerate(runs):
            assert m[g, p] == r.m
            np.testing.assert_allclose(alpha[g, p, :r.m], r.alpha, rtol=RTOL, atol=RTOL * lap.norm_bound())
            np.testing.assert_allclose(beta[g, p, :r.m - 1], r.beta, rtol=RTOL, atol=RTOL * lap.norm_bound())
            np.testing.assert_allclose(theta[g, p, :r.m], r.theta, rtol=RTOL, atol=RTOL * lap.norm_bound())
        oh, _ = odesc.heat_trace(runs, lap.n, t)
        # exp(-t theta) turns the eigensolver's absolute error eps * ||T|| into a
        # relative error t * ||L|| * eps: widen 1e-10 where that is larger
        # (combinatorial Laplacians with large degrees)
        rt = np.maximum(RTOL, t * lap.norm_bound() * 1e-14)
        assert np.all(np.abs(heat[g] - oh) <= rt * np.abs(oh)), g
        ov, _ = odesc.vnge(runs, lap.n, lap.trace)
        assert abs(vnge[g] - ov) <= RTOL * abs(ov) + 1e-300


def test_batch_equals_single_graph_runs():
    graphs = mixed_batch()
    nv, s, seed = 8, 12, 9
    gb = slaq.build_laplacian_batch(graphs)
    t = _dev(synth.t_grid(), torch.float64)
    for prec in (slaq.FP64, slaq.FP32):
        K = slaq.lanczos(gb, nv, s, seed, graph_id=3, precision=prec)
        hb = slaq.trace_heat(K, t)[0].cpu().numpy()
        for g, (src, dst, n) in enumerate(graphs):
            gs = slaq.build_laplacian(_dev(src, torch.int32), _dev(dst, torch.int32), n)
            Ks = slaq.lanczos(gs, nv, s, seed, graph_id=3 + g, precision=prec)
            hs = slaq.trace_heat(Ks, t)[0].cpu().numpy()
            tol = 1e-12 if prec == slaq.FP64 else 1e-5
            np.testing.assert_allclose(hb[g], hs, rtol=tol)


def test_weighted_batch():
    rng = np.random.default_rng(0)
    graphs = [synth.barabasi_albert(120, 2, seed=i) for i in range(4)]
    weights = [rng.uniform(0.5, 2.0, g[0].size) for g in graphs]
    gb = slaq.build_laplacian_batch(graphs, weights=weights, kind=slaq.COMBINATORIAL)
    K = slaq.lanczos(gb, 5, 8, 2)
    alpha = slaq.krylov_export(K)[0].cpu().numpy()
    for g, ((src, dst, n), w) in enumerate(zip(graphs, weights)):
        lap = build_laplacian(src, dst, n, weights=w, kind=COMBINATORIAL)
        runs = odesc.slq_runs(lap, 8, 5, 2, graph=g)
        for p, r in enumerate(runs):
            np.testing.assert_allclose(alpha[g, p, :r.m], r.alpha, rtol=RTOL)


def test_batch_rejects_bad_local_ids():
    graphs = [synth.path(5), (np.array([0, 7], np.int32), np.array([1, 2], np.int32), 4)]
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.build_laplacian_batch(graphs)
    assert ei.value.status == 1


def test_sbm_batch_reduced_precision():
    graphs = synth.sbm_batch(60, seed=3, median=80)
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    t = _dev(synth.t_grid(), torch.float64)
    h64 = slaq.trace_heat(slaq.lanczos(gb, 20, 15, 1, precision=slaq.FP64), t)[0].cpu().numpy()
    h32 = slaq.trace_heat(slaq.lanczos(gb, 20, 15, 1, precision=slaq.FP32), t)[0].cpu().numpy()
    assert np.max(np.abs(h32 - h64) / np.abs(h64)) < 1e-4


def many_small_graphs(count, seed=7):
    """A batch large enough (count x nv problems) for the thread-per-problem
    Gram solve: small BA, ER, cycle and star graphs of 12 to 60 nodes."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(12, 61))
        kind = i % 4
        if kind == 0:
            out.append(synth.barabasi_albert(n, 2, seed=seed + i))
        elif kind == 1:
            out.append(synth.erdos_renyi(n, 0.15, seed=seed + i))
        elif kind == 2:
            out.append(synth.cycle(n))
        else:
            out.append(synth.star(n))
    return out


@pytest.mark.parametrize("reorth", [1, 2])
def test_many_problems_solve_matches_oracle(reorth):
    graphs = many_small_graphs(272)
    nv, s, seed = 16, 10, 13          # 272 * 16 = 4352 problems per solve
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    K = slaq.lanczos(gb, nv, s, seed, precision=slaq.FP64, reorth_passes=reorth)
    alpha, beta, m = (x.cpu().numpy() for x in slaq.krylov_export(K))
    t = synth.t_grid(32)
    heat = slaq.trace_heat(K, _dev(t, torch.float64))[0].cpu().numpy()
    for g in range(0, len(graphs), 9):
        src, dst, n = graphs[g]
        lap = build_laplacian(src, dst, n, kind=NORMALIZED, drop_isolated=True)
        runs = odesc.slq_runs(lap, s, nv, seed, graph=g, reorth_passes=reorth)
        for p, r in enumerate(runs):
            assert m[g, p] == r.m, (g, p)
            np.testing.assert_allclose(alpha[g, p, :r.m], r.alpha, rtol=RTOL, atol=RTOL * lap.norm_bound())
            np.testing.assert_allclose(beta[g, p, :r.m - 1], r.beta, rtol=RTOL, atol=RTOL * lap.norm_bound())
        oh, _ = odesc.heat_trace(runs, lap.n, t)
        np.testing.assert_allclose(heat[g], oh, rtol=RTOL)
    # the FP32 solve of the reduced forms against the FP64 form
    h32 = slaq.trace_heat(slaq.lanczos(gb, nv, s, seed, precision=slaq.FP32, reorth_passes=reorth),
                          _dev(t, torch.float64))[0].cpu().numpy()
    assert np.max(np.abs(h32 - heat) / np.abs(heat)) < 1e-4


def _single_handles(graphs, kind=slaq.NORMALIZED, flags=0):
    return [slaq.build_laplacian(_dev(s, torch.int32), _dev(d, torch.int32), n, kind=kind, flags=flags)
            for s, d, n in graphs]


@pytest.mark.parametrize("prec", [slaq.FP64, slaq.FP32, slaq.FP32_BF16BASIS])
def test_lanczos_batched_equals_batch_build(prec):
    """The device-side concatenation of separately built graphs is the same
    block-diagonal Laplacian the batch builder makes, so the runs agree bit
    for bit."""
    graphs = mixed_batch()
    nv, s, seed = 6, 12, 21
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    want = slaq.krylov_export(slaq.lanczos(gb, nv, s, seed, graph_id=2, precision=prec))
    hs = _single_handles(graphs, flags=slaq.DROP_ISOLATED)
    K = slaq.lanczos_batched(hs, nv, s, seed, graph_id=2, precision=prec)
    del hs  # the Krylov handle owns the concatenation
    got = slaq.krylov_export(K)
    for a, b in zip(got, want):
        assert torch.equal(a, b)
    t_np = synth.t_grid()
    if prec == slaq.FP32_BF16BASIS:
        t_np = t_np[t_np <= 10.0]  # the t that form serves
    t = _dev(t_np, torch.float64)
    assert slaq.trace_heat(K, t)[0].shape == (len(graphs), t.numel())


def test_lanczos_batched_expands_batch_handles():
    graphs = mixed_batch()
    nv, s, seed = 5, 10, 3
    whole = slaq.build_laplacian_batch(graphs)
    parts = [slaq.build_laplacian_batch(graphs[:4]), *_single_handles(graphs[4:6]),
             slaq.build_laplacian_batch(graphs[6:])]
    a = slaq.krylov_export(slaq.lanczos(whole, nv, s, seed))
    b = slaq.krylov_export(slaq.lanczos_batched(parts, nv, s, seed))
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_lanczos_batched_tune_cache(tmp_path):
    graphs = mixed_batch()
    nv, s, seed = 8, 12, 4
    hs = _single_handles(graphs)
    cache = tmp_path / "tune.txt"
    K1 = slaq.lanczos_batched(hs, nv, s, seed, precision=slaq.FP64, tune_cache=str(cache))
    lines = [ln for ln in cache.read_text().splitlines() if ln and not ln.startswith("#")]
    assert len(lines) == 1 and "nv=8 s=12" in lines[0]
    shape = [int(x) for x in lines[0].split("|")[1].split()]
    assert len(shape) == 6 and shape[0] in (128, 256, 512) and shape[2] in (0, 64, 128, 256)
    assert shape[5] in (-1, 1)
    K2 = slaq.lanczos_batched(hs, nv, s, seed, precision=slaq.FP64, tune_cache=str(cache))
    assert cache.read_text().splitlines()[1:] == lines        # read, not re-tuned
    for x, y in zip(slaq.krylov_export(K1), slaq.krylov_export(K2)):
        assert torch.equal(x, y)
    # tuned launch shapes change only the rounding order
    ref = slaq.krylov_export(slaq.lanczos_batched(hs, nv, s, seed, precision=slaq.FP64))
    for x, y in zip(slaq.krylov_export(K1)[:2], ref[:2]):
        np.testing.assert_allclose(x.cpu().numpy(), y.cpu().numpy(), rtol=RTOL, atol=RTOL * 2)
    # every launch shape in the candidate lists runs correctly (TMA gathers in
    # the last field; a line of five fields, from before that field, reads as -1)
    for line in ("256 256 128 0 1 1", "512 128 64 128 0 -1", "128 512 256 256 1 1",
                 "256 256 0 0 -1 1", "256 256 128 0 1"):
        cache.write_text(lines[0].split("|")[0] + "| " + line + "\n")
        K3 = slaq.lanczos_batched(hs, nv, s, seed, precision=slaq.FP32, tune_cache=str(cache))
        h3 = slaq.trace_heat(K3, _dev(synth.t_grid(), torch.float64))[0].cpu().numpy()
        h64 = slaq.trace_heat(K1, _dev(synth.t_grid(), torch.float64))[0].cpu().numpy()
        assert np.max(np.abs(h3 - h64) / np.abs(h64)) < 1e-4, line


def test_lanczos_batched_rejects_mixed_kinds():
    graphs = mixed_batch()[:2]
    hs = _single_handles(graphs[:1]) + _single_handles(graphs[1:], kind=slaq.COMBINATORIAL)
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.lanczos_batched(hs, 4, 5, 1)
    assert ei.value.status == 1
    with pytest.raises(slaq.SlaqError):
        slaq.lanczos_batched([], 4, 5, 1)


@pytest.mark.parametrize("prec", [slaq.FP64, slaq.FP32])
def test_batch_graph_with_no_kept_nodes(prec):
    """A graph of a batch whose nodes are all isolated and dropped has an empty
    Krylov space: m = 0, zero traces and zero entropy, and the other graphs
    are unaffected."""
    empty = (np.zeros(0, np.int32), np.zeros(0, np.int32), 3)
    graphs = [synth.path(5), empty, synth.cycle(4)]
    nv, s, seed = 4, 6, 8
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    info = slaq.graph_batch_info(gb)
    assert list(np.diff(info["node_off"])) == [5, 0, 4]
    K = slaq.lanczos(gb, nv, s, seed, precision=prec)
    m = slaq.krylov_export(K)[2].cpu().numpy()
    assert np.all(m[1] == 0) and np.all(m[0] > 0) and np.all(m[2] > 0)
    t = _dev(synth.t_grid(32), torch.float64)
    heat = slaq.trace_heat(K, t)[0].cpu().numpy()
    vnge = slaq.trace_vnge(K)[0].cpu().numpy()
    (wr, _), _ = slaq.trace_wave(K, t)
    assert np.all(heat[1] == 0.0) and vnge[1] == 0.0 and np.all(wr[1].cpu().numpy() == 0.0)
    for g in (0, 2):
        src, dst, n = graphs[g]
        gs = slaq.build_laplacian(_dev(src, torch.int32), _dev(dst, torch.int32), n,
                                  flags=slaq.DROP_ISOLATED)
        hs = slaq.trace_heat(slaq.lanczos(gs, nv, s, seed, graph_id=g, precision=prec), t)[0]
        np.testing.assert_allclose(heat[g], hs.cpu().numpy(), rtol=1e-12 if prec == slaq.FP64 else 1e-5)


@pytest.mark.parametrize("precision", [slaq.FP32, slaq.FP32_BF16BASIS])
def test_batched_rayleigh_ritz_thread_per_problem_vs_fp64(precision):
    """>= 4096 problems take the thread-per-problem Rayleigh-Ritz kernel
    (the batch path); its rule must meet the reduced forms' bars against the
    FP64 form per graph: heat within relative 1e-4 on the t the form serves,
    VNGE within 1e-3."""
    graphs = synth.sbm_batch(220, seed=7)
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    nv, s = 20, 15
    assert 220 * nv >= 4096
    t_np = synth.t_grid(64)
    if precision == slaq.FP32_BF16BASIS:
        t_np = t_np[t_np * 2.0 <= 20.0]
    t = _dev(t_np, torch.float64)
    K64 = slaq.lanczos(gb, nv, s, 3, precision=slaq.FP64)
    K = slaq.lanczos(gb, nv, s, 3, precision=precision)
    h64 = slaq.trace_heat(K64, t)[0].cpu().numpy()
    h = slaq.trace_heat(K, t)[0].cpu().numpy()
    assert np.max(np.abs(h - h64) / np.abs(h64)) < 1e-4
    v64 = slaq.trace_vnge(K64)[0].cpu().numpy()
    v = slaq.trace_vnge(K)[0].cpu().numpy()
    assert np.max(np.abs(v - v64) / np.abs(v64)) < 1e-3
    if precision == slaq.FP32:
        # the FP32 form's own level: its Ritz values carry errors of about
        # ||L|| 2^-24, which exp(-t theta) turns into t ||L|| 2^-24 = 1.2e-5
        # relative at t = 100 (measured: 2.8e-6 heat, far less on VNGE)
        assert np.max(np.abs(h - h64) / np.abs(h64)) < 1e-5
        assert np.max(np.abs(v - v64) / np.abs(v64)) < 1e-5
