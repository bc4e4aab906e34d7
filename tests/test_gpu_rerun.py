"""slaq_lanczos_rerun: the handle's last Lanczos run replayed from a captured
CUDA graph with a new probe seed.  The replay issues the same kernels with
the same launch shapes on the same buffers, so it must equal a fresh
slaq_lanczos call with that seed bit for bit (coefficients, Gauss rules and
descriptors), for every form, for batches, and after the handle is reused."""
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


def _dev(a, dt=torch.int32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _graph(src, dst, n, drop=True):
    return slaq.build_laplacian(_dev(src), _dev(dst), n, flags=slaq.DROP_ISOLATED if drop else 0)


def _state(K):
    t_np = synth.t_grid(32)
    if slaq.krylov_info(K)["precision"] == slaq.FP32_BF16BASIS:
        t_np = t_np[t_np <= 10.0]  # the t that form serves
    t = _dev(t_np, torch.float64)
    return list(slaq.krylov_export(K)) + list(slaq.ritz_export(K)) + [slaq.trace_heat(K, t)[0]]


def _same(K, ref):
    for x, y in zip(_state(K), _state(ref)):
        assert torch.equal(x, y)


@pytest.mark.parametrize("prec", [slaq.FP64, slaq.FP32, slaq.FP32_BF16BASIS])
@pytest.mark.parametrize("reorth", [1, 2])
def test_rerun_equals_fresh_run(prec, reorth):
    src, dst, n = synth.rmat(13, 16 << 13, seed=3)     # split rows: both SpMM streams
    g = _graph(src, dst, n)
    nv, s = 17, 12
    K = slaq.lanczos(g, nv, s, 1, precision=prec, reorth_passes=reorth)
    for seed in (5, 9, 5):                               # capture, then replays
        slaq.lanczos_rerun(K, seed)
        _same(K, slaq.lanczos(g, nv, s, seed, precision=prec, reorth_passes=reorth))


def test_rerun_batches():
    graphs = [synth.barabasi_albert(300, 3, seed=1), synth.sbm([40, 40, 41], 0.3, 0.02, seed=2),
              synth.cycle(17), (np.zeros(0, np.int32), np.zeros(0, np.int32), 3),
              synth.rmat(11, 8 << 11, seed=4)]
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    K = slaq.lanczos(gb, 6, 10, 2, precision=slaq.FP32)
    for seed in (7, 8):
        slaq.lanczos_rerun(K, seed)
        _same(K, slaq.lanczos(gb, 6, 10, seed, precision=slaq.FP32))
    # a slaq_lanczos_batched handle owns its concatenation: the inputs may go
    hs = [_graph(*gr, drop=True) for gr in graphs[:3]]
    Kb = slaq.lanczos_batched(hs, 6, 10, 2, precision=slaq.FP64)
    ref = slaq.lanczos_batched(hs, 6, 10, 11, precision=slaq.FP64)
    for h in hs:
        h.close()
    slaq.lanczos_rerun(Kb, 11)
    _same(Kb, ref)


def test_rerun_after_reuse_and_errors():
    a = synth.barabasi_albert(500, 3, seed=2)
    b = synth.barabasi_albert(700, 2, seed=3)
    ga, gbb = _graph(*a), _graph(*b)
    K = slaq.lanczos(ga, 8, 10, 1, precision=slaq.FP64)
    slaq.lanczos_rerun(K, 4)
    # a new run on another graph discards the captured graph
    K = slaq.lanczos(gbb, 8, 10, 1, precision=slaq.FP64, reuse=K)
    slaq.lanczos_rerun(K, 6)
    _same(K, slaq.lanczos(gbb, 8, 10, 6, precision=slaq.FP64))
    # partial reorthogonalization decides on the host: not replayed
    Kp = slaq.lanczos(ga, 8, 10, 1, precision=slaq.FP64, reorth_passes=slaq.REORTH_PARTIAL)
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.lanczos_rerun(Kp, 2)
    assert ei.value.status == 6
    # the run's graph destroyed: refused before anything is launched
    gbb.close()
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.lanczos_rerun(K, 2)
    assert ei.value.status == 1


def test_batched_single_input_runs_in_place():
    """slaq_lanczos_batched with one handle runs on it without a copy: equal
    to slaq_lanczos on that handle bit for bit, replayable while the input
    lives, refused after it is destroyed."""
    graphs = synth.sbm_batch(12, seed=4)
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    Kb = slaq.lanczos_batched([gb], 6, 10, 3, precision=slaq.FP32)
    _same(Kb, slaq.lanczos(gb, 6, 10, 3, precision=slaq.FP32))
    slaq.lanczos_rerun(Kb, 5)
    _same(Kb, slaq.lanczos(gb, 6, 10, 5, precision=slaq.FP32))
    gb.close()
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.lanczos_rerun(Kb, 6)
    assert ei.value.status == 1
    # the traces of the completed run stay readable
    t = torch.as_tensor(synth.t_grid(8), device="cuda")
    assert torch.isfinite(slaq.trace_heat(Kb, t)[0]).all()
