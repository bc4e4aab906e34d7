"""Light-row SpMM through TMA row gathers (slaq_set_spmm_gathers) against the
load path and the FP64 form, through the C ABI.

The two gather paths do the same arithmetic in another summation order, so a
run through either must meet the reduced forms' bars against the FP64 run
(heat within relative 1e-4 on the t the form serves, VNGE within 1e-3), and
the two stay within a few units of their storage rounding of each other.
Covered: every row-group width of the kernel (one, two and four rows per
warp), every SpMM mode (pre-scaled gathers, scale gathers, weighted values),
split rows beside the TMA rows, rows without entries, a batch, the replay of
a TMA run from its CUDA graph, and the path's eligibility rules.
"""
import numpy as np
import pytest

import synth

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
    yield
    slaq.set_spmm_gathers(slaq.GATHERS_TUNED)


def _dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def _graph(edges, weights=None, drop=True):
    s, d, n = edges
    w = None if weights is None else _dev(weights, torch.float64)
    return slaq.build_laplacian(_dev(s, torch.int32), _dev(d, torch.int32), n, weights=w,
                                flags=slaq.DROP_ISOLATED if drop else 0)


def _served(t_np, precision):
    return t_np[t_np * 2.0 <= 20.0] if precision == slaq.FP32_BF16BASIS else t_np


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def _run(g, nv, s, seed, precision, mode):
    slaq.set_spmm_gathers(mode)
    K = slaq.lanczos(g, nv, s, seed, precision=precision)
    assert slaq.krylov_gathers(K) == (1 if mode == slaq.GATHERS_TMA else 0)
    return K


def _check(g, nv, s, seed, precision, close):
    t_np = _served(synth.t_grid(), precision)
    t = _dev(t_np, torch.float64)
    K64 = slaq.lanczos(g, nv, s, seed, precision=slaq.FP64)
    h64 = slaq.trace_heat(K64, t)[0].cpu().numpy()
    v64 = slaq.trace_vnge(K64)[0].item()
    Kt = _run(g, nv, s, seed, precision, slaq.GATHERS_TMA)
    Kl = _run(g, nv, s, seed, precision, slaq.GATHERS_LOADS)
    ht = slaq.trace_heat(Kt, t)[0].cpu().numpy()
    hl = slaq.trace_heat(Kl, t)[0].cpu().numpy()
    assert _rel(ht, h64) < 1e-4 and _rel(hl, h64) < 1e-4
    assert abs(slaq.trace_vnge(Kt)[0].item() - v64) / abs(v64) < 1e-3
    assert _rel(ht, hl) < close
    return Kt


# (nv, precision): 16-byte lanes per row 26 / 6 / 10 (FP32 nv = 100, 20, 37)
# and 8 / 14 / 26 (BF16 basis nv = 64, 100, 200) cover one, two and four rows
# per warp
@pytest.mark.parametrize("nv,precision,close", [
    (100, slaq.FP32, 1e-6), (20, slaq.FP32, 1e-6), (37, slaq.FP32, 1e-6),
    (64, slaq.FP32_BF16BASIS, 3e-5), (100, slaq.FP32_BF16BASIS, 3e-5),
    (200, slaq.FP32_BF16BASIS, 3e-5)])
def test_tma_rmat_with_split_rows(nv, precision, close):
    # R-MAT 2^13: hub rows above 2048 entries go to the split-row kernels
    g = _graph(synth.rmat(13, 16 << 13, seed=3))
    assert np.diff(slaq.graph_export(g)["rowptr"].cpu().numpy()).max() > 2048
    _check(g, nv, 12, 5, precision, close)


@pytest.mark.parametrize("precision", [slaq.FP32, slaq.FP32_BF16BASIS])
def test_tma_weighted_and_empty_rows(precision):
    # weighted values (the values form) and isolated nodes kept (rows
    # without entries inside the work items)
    s, d, n = synth.barabasi_albert(3000, 5, seed=12)
    w = np.random.default_rng(5).uniform(0.5, 2.0, s.size)
    _check(_graph((s, d, n), weights=w), 24, 16, 6, precision, 3e-5)
    isl = synth.disjoint_union(synth.erdos_renyi(300, 0.03, 1), synth.cycle(17), synth.star(40),
                               extra_isolated=9)
    _check(_graph(isl, drop=False), 33, 10, 2, precision, 3e-5)


@pytest.mark.parametrize("precision", [slaq.FP32, slaq.FP32_BF16BASIS])
def test_tma_batch(precision):
    graphs = synth.sbm_batch(60, seed=3)
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    t_np = _served(synth.t_grid(32), precision)
    t = _dev(t_np, torch.float64)
    h64 = slaq.trace_heat(slaq.lanczos(gb, 20, 15, 1, precision=slaq.FP64), t)[0].cpu().numpy()
    ht = slaq.trace_heat(_run(gb, 20, 15, 1, precision, slaq.GATHERS_TMA), t)[0].cpu().numpy()
    assert ht.shape == (60, t_np.size)
    assert _rel(ht, h64) < 1e-4


def test_tma_replay_and_reuse():
    g = _graph(synth.rmat(12, 16 << 12, seed=9))
    t = _dev(synth.t_grid(16), torch.float64)
    K = _run(g, 48, 10, 1, slaq.FP32, slaq.GATHERS_TMA)
    # the replay keeps the TMA path whatever the current mode
    slaq.set_spmm_gathers(slaq.GATHERS_LOADS)
    slaq.lanczos_rerun(K, 77)
    assert slaq.krylov_gathers(K) == 1
    h_replay = slaq.trace_heat(K, t)[0]
    K2 = _run(g, 48, 10, 77, slaq.FP32, slaq.GATHERS_TMA)
    assert torch.equal(slaq.trace_heat(K2, t)[0], h_replay)
    # deterministic: the same run twice is bit-identical
    K3 = _run(g, 48, 10, 77, slaq.FP32, slaq.GATHERS_TMA)
    for x, y in zip(slaq.krylov_export(K2), slaq.krylov_export(K3)):
        assert torch.equal(x, y)
    # a handle reused on a larger graph rebuilds its tensor map and work items
    g2 = _graph(synth.rmat(13, 16 << 13, seed=4))
    K4 = slaq.lanczos(g2, 48, 10, 3, precision=slaq.FP32, reuse=K3)
    K5 = _run(g2, 48, 10, 3, slaq.FP32, slaq.GATHERS_TMA)
    assert torch.equal(slaq.trace_heat(K4, t)[0], slaq.trace_heat(K5, t)[0])


def test_tma_eligibility():
    g = _graph(synth.barabasi_albert(500, 3, seed=1))
    # FP64 runs, and rows wider than a warp of 16-byte lanes, keep the loads
    assert _run_mode(g, 8, slaq.FP64) == 0
    assert _run_mode(g, 160, slaq.FP32) == 0          # 40 lanes of 16 bytes
    assert _run_mode(g, 128, slaq.FP32) == 1          # 32 lanes
    assert _run_mode(g, 256, slaq.FP32_BF16BASIS) == 1
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.set_spmm_gathers(2)
    assert ei.value.status == 1
    slaq.set_spmm_gathers(slaq.GATHERS_TUNED)


def _run_mode(g, nv, precision):
    slaq.set_spmm_gathers(slaq.GATHERS_TMA)
    K = slaq.lanczos(g, nv, 6, 1, precision=precision)
    return slaq.krylov_gathers(K)


def test_tma_wait_giveup_reports_timeout():
    """The bounded-wait error path (slaq_debug_tma_giveup): every warp's first
    stage wait gives up, the kernel drains its copies and flags the run, which
    returns SLAQ_ETIMEOUT and leaves the handle not ready; the next run on the
    handle is bit-equal to the one before; the load path ignores the hook."""
    g = _graph(synth.rmat(12, 16 << 12, seed=9))
    t = _dev(synth.t_grid(16), torch.float64)
    K = _run(g, 32, 8, 1, slaq.FP32, slaq.GATHERS_TMA)
    want = slaq.trace_heat(K, t)[0].clone()
    slaq.debug_tma_giveup(True)
    try:
        with pytest.raises(slaq.SlaqError) as ei:
            slaq.lanczos(g, 32, 8, 1, precision=slaq.FP32, reuse=K)
        assert ei.value.status == 5  # SLAQ_ETIMEOUT
        with pytest.raises(slaq.SlaqError) as ei:
            slaq.trace_heat(K, t)
        assert ei.value.status == 1
        slaq.set_spmm_gathers(slaq.GATHERS_LOADS)
        Kl = slaq.lanczos(g, 32, 8, 1, precision=slaq.FP32)
        assert slaq.krylov_gathers(Kl) == 0
    finally:
        slaq.debug_tma_giveup(False)
    K2 = _run(g, 32, 8, 1, slaq.FP32, slaq.GATHERS_TMA)
    assert torch.equal(slaq.trace_heat(K2, t)[0], want)
    K3 = slaq.lanczos(g, 32, 8, 1, precision=slaq.FP32, reuse=K)
    assert torch.equal(slaq.trace_heat(K3, t)[0], want)
