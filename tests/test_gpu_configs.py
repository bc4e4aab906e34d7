"""The web-scale and graph-pair workloads as parity cases, through the C ABI.

* R-MAT 2^24 with 16 * 2^24 unique undirected edges (a, b, c, d = .57, .19,
  .19, .05), isolated nodes dropped, normalized Laplacian, nv = 64, s = 20.
  Too large for the oracle, the FP64 run is held to invariants that hold at
  any size (the Gauss rules' first two moments against q^T L q and ||L q||^2
  of a direct sparse product, h(0) = n'), and
  the BF16-basis form (and the FP32 form) against the FP64 form on the same
  probes.  The FP64 run takes the first 32 probes, whose basis alone is
  46 GB (nv = 64 would double it); every probe's Lanczos run is independent
  of the others, so the mean over probes 0..31 of the nv = 64 run is the
  nv = 32 estimate.  Bars: relative 1e-4 on the heat trace, 1e-3 on the
  VNGE, and 1e-4 of the largest |Re| on the wave trace.  The BF16-basis form
  serves its heat and wave traces for t * bound <= 20 only (t <= 10 here; the
  library refuses larger t): beyond it the first-order sensitivity of the
  unconverged Ritz values to the basis rounding grows with t (the wave trace
  measured 0.28 off at t = 100; the heat trace of this graph stays within
  1e-4, but that of graphs with many small eigenvalues does not).
* Graph pairs: R-MAT graphs of 2^14 .. 2^17 nodes (16 edges per node), each
  against a copy with 0.1% of its edges rewired, nodes kept (no dropping), as
  two batches whose graph g shares probe graph field g (common random
  probes).  FP64 distances equal the oracle's on the smallest pair within
  1e-10 of the descriptors' size (the per-entry bar, carried through the
  cancelling difference);
  the reduced forms' heat and VNGE distances are within relative 1e-3 of
  FP64's, wave distances within 1e-2 (the BF16 basis over the t <= 10 it
  serves, as above).
* The 5000-graph SBM batch at full size (sizes lognormal, median 300, seed
  3; isolated nodes dropped; nv = 20, s = 15, probe seed 1) through
  slaq_lanczos_batched on the batch handle, as the bench runs it: FP64
  coefficients and heat traces of sampled graphs (the largest, the smallest
  and every 500th) equal the oracle's for that graph alone within relative
  1e-10; every graph's FP32 heat trace within 1e-4 of FP64 and its VNGE
  within 1e-3 (absolute where the VNGE is below 1).
"""
import warnings

import numpy as np
import pytest

import synth
from oracle import descriptors as odesc
from oracle import distance as odist
from oracle.laplacian import NORMALIZED, build_laplacian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2003_01282_gb300 import slaq  # noqa: E402
from paper_2003_01282_gb300.build import build  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build()
    slaq.lib()


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def test_rmat24_reduced_forms_vs_fp64():
    src, dst, n = synth.rmat_torch(24, 16 << 24, seed=2)
    g = slaq.build_laplacian(src, dst, n, flags=slaq.DROP_ISOLATED)
    del src, dst
    info = g.info
    assert info["nnz"] == 2 * (16 << 24) and info["trace"] == info["n"]
    t = torch.as_tensor(synth.t_grid(), device="cuda")
    K64 = slaq.lanczos(g, 32, 20, 2, precision=slaq.FP64)
    h64 = slaq.trace_heat(K64, t)[0].cpu().numpy()
    v64 = slaq.trace_vnge(K64)[0].item()
    (w64, _), _ = slaq.trace_wave(K64, t)
    w64 = w64.cpu().numpy()
    _check_moments(g, K64, 32, seed=2)
    del K64
    t_np = synth.t_grid()
    lo = t_np <= 10.0
    t_lo = t[torch.as_tensor(lo, device="cuda")].contiguous()   # the t the BF16 basis serves
    # the BF16-basis form at the workload's nv = 64, first 32 probes
    Kb = slaq.lanczos(g, 64, 20, 2, precision=slaq.FP32_BF16BASIS)
    _, _, hp = slaq.trace_heat(Kb, t_lo, per_probe=True)
    _, _, vp = slaq.trace_vnge(Kb, per_probe=True)
    assert _rel(hp[:32].mean(0).cpu().numpy(), h64[lo]) < 1e-4
    assert abs(vp[:32].mean().item() - v64) / v64 < 1e-3
    del Kb
    for prec in (slaq.FP32_BF16BASIS, slaq.FP32):
        K = slaq.lanczos(g, 32, 20, 2, precision=prec)
        ts, sel = (t_lo, lo) if prec == slaq.FP32_BF16BASIS else (t, np.ones_like(lo))
        h = slaq.trace_heat(K, ts)[0].cpu().numpy()
        assert _rel(h, h64[sel]) < 1e-4, prec
        (w, _), _ = slaq.trace_wave(K, ts)
        werr = np.abs(w.cpu().numpy() - w64[sel])
        assert np.max(werr) < 1e-4 * np.max(np.abs(w64)), prec
        assert abs(slaq.trace_vnge(K)[0].item() - v64) / v64 < 1e-3, prec
        del K


def _check_moments(g, K, nv, seed):
    """Invariants of the FP64 run that hold at any size: the Gauss rule of
    probe q is exact for polynomials up to degree 2m - 1, so its first two
    moments equal q^T L q / q^T q and ||L q||^2 / q^T q, computed here from
    the exported CSR and probes by one FP64 sparse product (cuSPARSE through
    torch), independently of the Lanczos kernels; and h(0) = n' (the
    weights of every probe sum to one)."""
    ex = slaq.graph_export(g)
    n = g.info["n"]
    with warnings.catch_warnings():  # torch marks sparse CSR tensors as beta
        warnings.simplefilter("ignore", UserWarning)
        A = torch.sparse_csr_tensor(ex["rowptr"], ex["colidx"].to(torch.int64), ex["vals"],
                                    size=(n, n))
    q = slaq.probes(g, nv, seed)
    y = torch.matmul(A, q) + ex["diag"][:n, None] * q
    del A, ex
    qq = (q * q).sum(0)
    m1 = ((q * y).sum(0) / qq).cpu().numpy()
    m2 = ((y * y).sum(0) / qq).cpu().numpy()
    del q, y
    theta, tau2 = slaq.ritz_export(K)
    g1 = (tau2 * theta).sum(1).cpu().numpy()
    g2 = (tau2 * theta * theta).sum(1).cpu().numpy()
    assert np.max(np.abs(g1 - m1) / np.abs(m1)) < 1e-10
    assert np.max(np.abs(g2 - m2) / np.abs(m2)) < 1e-10
    h0 = slaq.trace_heat(K, torch.zeros(1, dtype=torch.float64, device="cuda"))[0].item()
    assert abs(h0 - n) <= 1e-12 * n


def _pairs():
    orig, copy = [], []
    for i, scale in enumerate((14, 15, 16, 17)):
        s, d, n = synth.rmat(scale, 16 << scale, seed=100 + i)
        s2, d2, _ = synth.rewire(s, d, n, frac=1e-3, seed=i)
        orig.append((s, d, n))
        copy.append((s2, d2, n))
    return orig, copy


def _descriptors(handles, prec, t):
    K = slaq.lanczos_batched(handles, 64, 20, 5, precision=prec)
    heat = slaq.trace_heat(K, t)[0]
    (wr, _), (wi, _) = slaq.trace_wave(K, t)
    vn = slaq.trace_vnge(K)[0]
    return heat, wr, wi, vn


def test_graph_pair_distances():
    orig, copy = _pairs()
    t_np = synth.t_grid()
    t = torch.as_tensor(t_np, device="cuda")
    ha = [slaq.build_laplacian(torch.as_tensor(s, device="cuda"), torch.as_tensor(d, device="cuda"), n)
          for s, d, n in orig]
    hb = [slaq.build_laplacian(torch.as_tensor(s, device="cuda"), torch.as_tensor(d, device="cuda"), n)
          for s, d, n in copy]
    dist = {}
    lo_np = t_np <= 10.0
    lo = torch.as_tensor(lo_np, device="cuda")
    nlo = int(lo_np.sum())
    for prec in (slaq.FP64, slaq.FP32, slaq.FP32_BF16BASIS):
        # the BF16-basis form serves its traces for t <= 10 only
        ts = t[lo].contiguous() if prec == slaq.FP32_BF16BASIS else t
        A, B = _descriptors(ha, prec, ts), _descriptors(hb, prec, ts)
        out = []
        for i in range(len(orig)):
            # whole grid (nan where the form does not serve it) and t <= 10
            full = prec != slaq.FP32_BF16BASIS
            dh = slaq.distance(A[0][i], B[0][i], slaq.DIST_HEAT).item() if full else float("nan")
            dw = slaq.distance(torch.cat([A[1][i], A[2][i]]), torch.cat([B[1][i], B[2][i]]),
                               slaq.DIST_WAVE).item() if full else float("nan")
            dhl = slaq.distance(A[0][i][:nlo].contiguous(), B[0][i][:nlo].contiguous(),
                                slaq.DIST_HEAT).item()
            dwl = slaq.distance(torch.cat([A[1][i][:nlo], A[2][i][:nlo]]),
                                torch.cat([B[1][i][:nlo], B[2][i][:nlo]]), slaq.DIST_WAVE).item()
            dv = slaq.distance(A[3][i:i + 1], B[3][i:i + 1], slaq.DIST_VNGE).item()
            out.append((dh, dw, dv, dwl, dhl))
        dist[prec] = np.array(out)
        if prec == slaq.FP64:
            # the smallest pair against the oracle, same probes (graph field 0)
            (sa, da, n), (sb, db, _) = orig[0], copy[0]
            la = build_laplacian(sa, da, n, kind=NORMALIZED)
            lb = build_laplacian(sb, db, n, kind=NORMALIZED)
            ra, rb = odesc.slq_runs(la, 20, 64, 5, graph=0), odesc.slq_runs(lb, 20, 64, 5, graph=0)
            oha, _ = odesc.heat_trace(ra, la.n, t_np)
            ohb, _ = odesc.heat_trace(rb, lb.n, t_np)
            (owra, _), (owia, _) = odesc.wave_trace(ra, la.n, t_np)
            (owrb, _), (owib, _) = odesc.wave_trace(rb, lb.n, t_np)
            ova, _ = odesc.vnge(ra, la.n, la.trace)
            ovb, _ = odesc.vnge(rb, lb.n, lb.trace)
            want = (odist.heat_distance(oha, ohb), odist.wave_distance(owra, owia, owrb, owib),
                    odist.vnge_distance(ova, ovb))
            # a distance between nearby descriptors cancels: the 1e-10 bar per
            # descriptor entry carries over to the distance relative to the
            # descriptors' own size, not to the (0.1%-small) distance
            scale = (np.linalg.norm(oha) + np.linalg.norm(ohb),
                     np.linalg.norm(np.concatenate([owra, owia])) +
                     np.linalg.norm(np.concatenate([owrb, owib])),
                     abs(ova) + abs(ovb))
            for k in range(3):
                assert abs(out[0][k] - want[k]) <= 1e-10 * scale[k], (k, out[0][k], want[k])
    for prec in (slaq.FP32, slaq.FP32_BF16BASIS):
        hcol, wcol = (0, 1) if prec == slaq.FP32 else (4, 3)
        assert _rel(dist[prec][:, [hcol, 2]], dist[slaq.FP64][:, [hcol, 2]]) < 1e-3, prec
        assert _rel(dist[prec][:, wcol], dist[slaq.FP64][:, wcol]) < 1e-2, prec


def test_sbm5000_batch_full_size_sampled_graphs():
    graphs = synth.sbm_batch(5000, seed=3)
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    nv, s, seed = 20, 15, 1
    t_np = synth.t_grid(64)
    t = torch.as_tensor(t_np, device="cuda", dtype=torch.float64)
    K64 = slaq.lanczos_batched([gb], nv, s, seed, precision=slaq.FP64)
    K32 = slaq.lanczos_batched([gb], nv, s, seed, precision=slaq.FP32)
    h64 = slaq.trace_heat(K64, t)[0].cpu().numpy()
    h32 = slaq.trace_heat(K32, t)[0].cpu().numpy()
    v64 = slaq.trace_vnge(K64)[0].cpu().numpy()
    v32 = slaq.trace_vnge(K32)[0].cpu().numpy()
    assert h64.shape == (5000, 64)
    # every graph: the FP32 form against FP64
    assert _rel(h32, h64) < 1e-4
    # VNGE: relative 1e-3, absolute below 1 (a graph left with one edge has
    # VNGE exactly 0, where a relative bar means nothing)
    assert np.all(np.abs(v32 - v64) <= 1e-3 * np.maximum(np.abs(v64), 1.0))
    # sampled graphs one by one against the oracle
    alpha, beta, m = (x.cpu().numpy() for x in slaq.krylov_export(K64))
    sizes = np.array([g[2] for g in graphs])
    sample = sorted({int(sizes.argmax()), int(sizes.argmin()), *range(0, 5000, 500)})
    for g in sample:
        src, dst, n = graphs[g]
        lap = build_laplacian(src, dst, n, drop_isolated=True)
        runs = odesc.slq_runs(lap, s, nv, seed, graph=g)
        for p, r in enumerate(runs):
            assert m[g, p] == r.m
            np.testing.assert_allclose(alpha[g, p, :r.m], r.alpha, rtol=1e-10, atol=1e-12)
        want, _ = odesc.heat_trace(runs, lap.n, t_np)
        assert _rel(h64[g], want) < 1e-10, g
