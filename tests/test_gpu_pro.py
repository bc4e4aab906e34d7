"""Partial reorthogonalization (slaq_lanczos with reorth_passes =
SLAQ_REORTH_PARTIAL) through the C ABI.

The GPU decides per graph, one step ahead, from every probe's omega
estimates, and projects partial steps on u_{k-1}, u_k with their 2 x 2 Gram
matrix; the oracle (oracle/lanczos.py ``lanczos_partial``) is the textbook
per-probe form.  Both keep the basis semi-orthogonal, so both give the Gauss
rule of full reorthogonalization to working accuracy.  The FP64 form is held
to relative 1e-10 against the oracle with full AND with partial
reorthogonalization on m, on alpha and beta up to the oracle's first
reorthogonalized step, and on the heat trace, the VNGE and the wave trace
for t < 10.  Past that step the T entries themselves are not comparable
entry by entry: once Ritz values have converged the continuation of the
recurrence is decided by rounding (on R-MAT 2^13 the oracle's own full and
partial runs differ by 0.3 in alpha_30..39 at s = 40, while their heat traces
agree to 3e-15 and both equal the exact q0^T e^{-tL} q0 to 1e-13).  The
unconverged tail of the wave trace (t >= 10) depends on those entries; there
the bar is 1e-5 of max |Re| (the oracle's two forms differ by 1.7e-7).
The FP32 form is held to 1e-4 (heat) and 1e-3 (VNGE) of the FP64 form."""
import numpy as np
import pytest

import synth
from oracle import descriptors as odesc
from oracle import lanczos as olz
from oracle import probes as oprobes
from oracle.laplacian import COMBINATORIAL, NORMALIZED, build_laplacian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2003_01282_gb300 import slaq  # noqa: E402
from paper_2003_01282_gb300.build import build  # noqa: E402

RTOL = 1e-10
PARTIAL = slaq.REORTH_PARTIAL


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build()
    slaq.lib()


def _dev(a, dt=torch.int32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _graph(src, dst, n, kind=NORMALIZED, drop=False, w=None):
    return slaq.build_laplacian(_dev(src), _dev(dst), n,
                                weights=None if w is None else _dev(w, torch.float64),
                                kind=slaq.NORMALIZED if kind == NORMALIZED else slaq.COMBINATORIAL,
                                flags=slaq.DROP_ISOLATED if drop else 0)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


CASES = {
    # name: (generator, kind, drop isolated, weight seed, nv, s)
    "ba2000": (lambda: synth.barabasi_albert(2000, 4, seed=0), NORMALIZED, False, None, 10, 40),
    "ba2000_comb": (lambda: synth.barabasi_albert(2000, 4, seed=0), COMBINATORIAL, False, None, 7, 40),
    "rmat13": (lambda: synth.rmat(13, 16 << 13, seed=3), NORMALIZED, True, None, 17, 40),
    "islands": (lambda: synth.disjoint_union(synth.erdos_renyi(300, 0.03, 1), synth.cycle(17),
                                             synth.star(40), extra_isolated=9),
                NORMALIZED, False, None, 33, 30),
    "k9": (lambda: synth.complete(9), NORMALIZED, False, None, 6, 8),          # breakdown, m = 2
    "star30": (lambda: synth.star(30), COMBINATORIAL, False, None, 5, 8),      # breakdown, m = 3
    "ba600_w": (lambda: synth.barabasi_albert(600, 3, seed=8), NORMALIZED, False, 3, 9, 30),
    "ba600_w_comb": (lambda: synth.barabasi_albert(600, 3, seed=8), COMBINATORIAL, False, 3, 9, 30),
}


def _descriptors_close(K, runs, lap, t):
    td = _dev(t, torch.float64)
    h = slaq.trace_heat(K, td)[0].cpu().numpy()
    oh, _ = odesc.heat_trace(runs, lap.n, t)
    # exp(-t theta) turns the eigensolver's absolute error into t ||L|| eps relative
    bar = np.maximum(RTOL, t * lap.norm_bound() * 1e-14)
    assert np.all(np.abs(h - oh) <= bar * np.abs(oh))
    (wr, _), (wi, _) = slaq.trace_wave(K, td)
    (owr, _), (owi, _) = odesc.wave_trace(runs, lap.n, t)
    lo = t < 10
    for a, b in ((wr.cpu().numpy(), owr), (wi.cpu().numpy(), owi)):
        scale = np.max(np.abs(owr))
        assert np.max(np.abs(a - b)[lo]) < RTOL * scale
        assert np.max(np.abs(a - b)) < 1e-5 * scale
    v = slaq.trace_vnge(K)[0].item()
    ov, _ = odesc.vnge(runs, lap.n, lap.trace)
    assert abs(v - ov) <= RTOL * abs(ov) + 1e-300


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_partial_matches_oracle(name):
    gen, kind, drop, wseed, nv, s = CASES[name]
    src, dst, n = gen()
    w = None if wseed is None else np.random.default_rng(wseed).uniform(0.5, 2.0, src.size)
    lap = build_laplacian(src, dst, n, weights=w, kind=kind, drop_isolated=drop)
    g = _graph(src, dst, n, kind, drop, w)
    seed = 11
    K = slaq.lanczos(g, nv, s, seed, precision=slaq.FP64, reorth_passes=PARTIAL)
    alpha, beta, m = (x.cpu().numpy() for x in slaq.krylov_export(K))
    theta, _ = (x.cpu().numpy() for x in slaq.ritz_export(K))
    t = synth.t_grid(64)
    bound = lap.norm_bound()
    L = lap.matrix()
    # the oracle's first reorthogonalized step, per probe (m - 1 if none)
    first, triggered = [], []
    for p in range(nv):
        r = olz.lanczos_partial(L, oprobes.rademacher(seed, 0, p, lap.old_id), s, bound)
        first.append(r.full_steps[0] if r.full_steps else r.m - 1)
        # the GPU flags step k + 2 where the oracle reorthogonalizes at step k
        # (it learns beta from the next Gram diagonal): count the probes for
        # which that step still forms a vector (not at a breakdown)
        if r.full_steps and r.full_steps[0] + 2 < min(r.m, s - 1):
            triggered.append(r.full_steps[0])
    for partial in (False, True):
        runs = odesc.slq_runs(lap, s, nv, seed, partial=partial)
        for p, r in enumerate(runs):
            assert m[p] == r.m, (p, m[p], r.m)
            kf = first[p] + 1
            np.testing.assert_allclose(alpha[p, :kf], r.alpha[:kf], rtol=RTOL, atol=RTOL * bound)
            np.testing.assert_allclose(beta[p, :kf - 1], r.beta[:kf - 1], rtol=RTOL,
                                       atol=RTOL * bound)
            if r.m <= 12:  # short runs: every Ritz value is converged
                np.testing.assert_allclose(theta[p, :r.m], r.theta, rtol=RTOL, atol=RTOL * bound)
        _descriptors_close(K, runs, lap, t)
    full = slaq.krylov_full_steps(K).cpu().numpy()
    formed = min(int(m.max()), s - 1)
    assert np.all(full[:min(2, formed)] == 1) and np.all(full[formed:] == 0)
    assert full[2:].sum() <= s // 2, full
    if triggered:
        assert full[2:].sum() >= 1, (full, triggered)


def test_fp32_partial_vs_fp64():
    src, dst, n = synth.rmat(13, 16 << 13, seed=3)
    g = _graph(src, dst, n, drop=True)
    t = _dev(synth.t_grid(), torch.float64)
    K64 = slaq.lanczos(g, 32, 30, 9, precision=slaq.FP64)
    h64 = slaq.trace_heat(K64, t)[0].cpu().numpy()
    v64 = slaq.trace_vnge(K64)[0].item()
    K = slaq.lanczos(g, 32, 30, 9, precision=slaq.FP32, reorth_passes=PARTIAL)
    assert _rel(slaq.trace_heat(K, t)[0].cpu().numpy(), h64) < 1e-4
    assert abs(slaq.trace_vnge(K)[0].item() - v64) / abs(v64) < 1e-3
    # FP32 reaches sqrt(eps) sooner: more full steps than FP64, still not all
    K64p = slaq.lanczos(g, 32, 30, 9, precision=slaq.FP64, reorth_passes=PARTIAL)
    f32 = slaq.krylov_full_steps(K).cpu().numpy()[2:].sum()
    f64 = slaq.krylov_full_steps(K64p).cpu().numpy()[2:].sum()
    assert f64 <= f32 < 27, (f64, f32)


def test_partial_batch_per_graph():
    empty = (np.zeros(0, np.int32), np.zeros(0, np.int32), 4)
    graphs = [synth.barabasi_albert(900, 3, seed=1), synth.sbm([60, 60, 61], 0.3, 0.02, seed=2),
              empty, synth.cycle(17), synth.rmat(11, 8 << 11, seed=4)]
    nv, s, seed = 8, 30, 5
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    K = slaq.lanczos(gb, nv, s, seed, precision=slaq.FP64, reorth_passes=PARTIAL)
    t = _dev(synth.t_grid(32), torch.float64)
    heat = slaq.trace_heat(K, t)[0].cpu().numpy()
    full = slaq.krylov_full_steps(K).cpu().numpy()
    m = slaq.krylov_export(K)[2].cpu().numpy()
    assert np.all(m[2] == 0) and np.all(heat[2] == 0.0) and np.all(full[2] == 0)
    for gi, (src, dst, n) in enumerate(graphs):
        if gi == 2:
            continue
        gs = _graph(src, dst, n, drop=True)
        Ks = slaq.lanczos(gs, nv, s, seed, graph_id=gi, precision=slaq.FP64, reorth_passes=PARTIAL)
        np.testing.assert_allclose(heat[gi], slaq.trace_heat(Ks, t)[0].cpu().numpy(), rtol=1e-12)
        # per-graph decisions: the same steps as the graph alone
        assert np.array_equal(full[gi], slaq.krylov_full_steps(Ks).cpu().numpy()), gi
        lap = build_laplacian(src, dst, n, drop_isolated=True)
        runs = odesc.slq_runs(lap, s, nv, seed, graph=gi)
        oh, _ = odesc.heat_trace(runs, lap.n, synth.t_grid(32))
        bar = np.maximum(RTOL, synth.t_grid(32) * lap.norm_bound() * 1e-14)
        assert np.all(np.abs(heat[gi] - oh) <= bar * np.abs(oh)), gi


def test_partial_many_problems_thread_solve():
    """>= 4096 (graph, probe) problems: the thread-per-problem solve."""
    rng = np.random.default_rng(7)
    graphs = []
    for i in range(272):
        nn = int(rng.integers(40, 90))
        graphs.append(synth.barabasi_albert(nn, 2, seed=100 + i) if i % 2 == 0
                      else synth.erdos_renyi(nn, 0.12, seed=100 + i))
    nv, s, seed = 16, 24, 13
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    K = slaq.lanczos(gb, nv, s, seed, precision=slaq.FP64, reorth_passes=PARTIAL)
    alpha, beta, m = (x.cpu().numpy() for x in slaq.krylov_export(K))
    t = synth.t_grid(32)
    heat = slaq.trace_heat(K, _dev(t, torch.float64))[0].cpu().numpy()
    for gi in range(0, len(graphs), 17):
        src, dst, n = graphs[gi]
        lap = build_laplacian(src, dst, n, drop_isolated=True)
        runs = odesc.slq_runs(lap, s, nv, seed, graph=gi)
        for p, r in enumerate(runs):
            assert m[gi, p] == r.m, (gi, p)
        oh, _ = odesc.heat_trace(runs, lap.n, t)
        bar = np.maximum(RTOL, t * lap.norm_bound() * 1e-14)
        assert np.all(np.abs(heat[gi] - oh) <= bar * np.abs(oh)), gi


def test_full_steps_export_and_errors():
    src, dst, n = synth.barabasi_albert(500, 3, seed=2)
    g = _graph(src, dst, n)
    K = slaq.lanczos(g, 4, 12, 1, precision=slaq.FP64)
    full = slaq.krylov_full_steps(K).cpu().numpy()
    assert np.array_equal(full, np.r_[np.ones(11, np.int32), 0])
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.lanczos(g, 4, 12, 1, precision=slaq.FP32_BF16BASIS, reorth_passes=PARTIAL)
    assert ei.value.status == 6
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.lanczos(g, 4, 12, 1, precision=slaq.FP64, reorth_passes=3)
    assert ei.value.status == 1
    # a handle reused across modes: partial after full, full after partial
    K = slaq.lanczos(g, 4, 12, 1, precision=slaq.FP64, reorth_passes=PARTIAL, reuse=K)
    K2 = slaq.lanczos(g, 4, 12, 1, precision=slaq.FP64)
    K = slaq.lanczos(g, 4, 12, 1, precision=slaq.FP64, reuse=K)
    t = _dev(synth.t_grid(16), torch.float64)
    assert torch.equal(slaq.trace_heat(K, t)[0], slaq.trace_heat(K2, t)[0])


def test_partial_full_size_workload():
    """R-MAT 2^20, 16M edges, nv = 100, s = 20: FP64 with partial
    reorthogonalization against the oracle on two sampled probes, FP32 with
    it against the FP64 form with full reorthogonalization."""
    src, dst, n = synth.rmat(20, 16 << 20, seed=1)
    lap = build_laplacian(src, dst, n, drop_isolated=True)
    g = _graph(src, dst, n, drop=True)
    K64p = slaq.lanczos(g, 100, 20, 1, precision=slaq.FP64, reorth_passes=PARTIAL)
    alpha, beta, m = (x.cpu().numpy() for x in slaq.krylov_export(K64p))
    L = lap.matrix()
    for p in (0, 61):
        r = olz.lanczos_partial(L, oprobes.rademacher(1, 0, p, lap.old_id), 20, 2.0)
        assert m[p] == r.m
        kf = (r.full_steps[0] if r.full_steps else r.m - 1) + 1
        np.testing.assert_allclose(alpha[p, :kf], r.alpha[:kf], rtol=RTOL, atol=RTOL * 2)
        np.testing.assert_allclose(beta[p, :kf - 1], r.beta[:kf - 1], rtol=RTOL, atol=RTOL * 2)
    t = _dev(synth.t_grid(), torch.float64)
    K64 = slaq.lanczos(g, 100, 20, 1, precision=slaq.FP64)
    h64 = slaq.trace_heat(K64, t)[0].cpu().numpy()
    v64 = slaq.trace_vnge(K64)[0].item()
    assert _rel(slaq.trace_heat(K64p, t)[0].cpu().numpy(), h64) < 1e-10
    K32p = slaq.lanczos(g, 100, 20, 1, precision=slaq.FP32, reorth_passes=PARTIAL)
    assert _rel(slaq.trace_heat(K32p, t)[0].cpu().numpy(), h64) < 1e-4
    assert abs(slaq.trace_vnge(K32p)[0].item() - v64) / v64 < 1e-3


@pytest.mark.parametrize("prec,h_tol", [(slaq.FP64, 1e-10), (slaq.FP32, 1e-4)])
def test_partial_near_breakdown_probes(prec, h_tol):
    """SBM graphs 800..899 of the 5000-graph batch (probe seed 1, nv = 20,
    s = 15; graph_id 800 gives each graph the probes it has in the full
    batch).  Some probes of graphs 853 and 872 come within a factor 1.3 of the
    breakdown tolerance (beta_8 = 2.6e-4 in FP32), which leaves their next
    vector far from orthogonal before the one-step-late flag takes effect.
    A full step must stay finite there; the descriptors hold the form's bar
    against full reorthogonalization in FP64."""
    graphs = synth.sbm_batch(5000, seed=3)[800:900]
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    t = _dev(synth.t_grid(64), torch.float64)
    Kp = slaq.lanczos(gb, 20, 15, 1, graph_id=800, precision=prec, reorth_passes=PARTIAL)
    alpha, beta, m = (x.cpu().numpy() for x in slaq.krylov_export(Kp))
    for g in range(len(graphs)):
        for p in range(20):
            assert np.all(np.isfinite(alpha[g, p, :m[g, p]])), (g, p)
            assert np.all(np.isfinite(beta[g, p, :max(m[g, p] - 1, 0)])), (g, p)
    K64 = slaq.lanczos(gb, 20, 15, 1, graph_id=800, precision=slaq.FP64)
    h, h64 = (slaq.trace_heat(K, t)[0].cpu().numpy() for K in (Kp, K64))
    keep = h64 > 0  # graphs with no kept nodes have a zero trace in both
    assert np.max(np.abs(h - h64)[keep] / h64[keep]) < h_tol


@pytest.mark.parametrize("nv,s", [(512, 6), (3, 64)])
def test_partial_largest_sizes(nv, s):
    """Partial reorthogonalization at the largest probe block and step count:
    the omega ring and the step flags span s + 2 entries."""
    src, dst, n = synth.barabasi_albert(2000, 4, seed=0)
    lap = build_laplacian(src, dst, n)
    g = _graph(src, dst, n)
    K = slaq.lanczos(g, nv, s, 11, precision=slaq.FP64, reorth_passes=PARTIAL)
    m = slaq.krylov_export(K)[2].cpu().numpy()
    runs = odesc.slq_runs(lap, s, nv, 11)
    assert all(m[p] == r.m for p, r in enumerate(runs))
    _descriptors_close(K, runs, lap, synth.t_grid(64))
    full = slaq.krylov_full_steps(K).cpu().numpy()
    assert full.shape == (s,) and full[:2].sum() == 2 and full[s - 1] == 0
