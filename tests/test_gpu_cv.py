"""The heat trace with the polynomial control variate, through the C ABI,
against the oracle (oracle/variance.py) on the same probes: FP64 within
relative 1e-10 per entry (estimate and standard error), reduced forms within
1e-4 of the FP64 form, batches per graph, and the variance reduction itself."""
import numpy as np
import pytest

import synth
from oracle import descriptors as odesc
from oracle import variance as ovar
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


def _dev(a, dt=torch.int32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


CASES = {
    "ba2000": (lambda: synth.barabasi_albert(2000, 4, seed=0), NORMALIZED, False, None),
    "rmat13": (lambda: synth.rmat(13, 16 << 13, seed=3), NORMALIZED, True, None),
    "islands": (lambda: synth.disjoint_union(synth.erdos_renyi(300, 0.03, 1), synth.cycle(17),
                                              extra_isolated=9), NORMALIZED, False, None),
    "ba_comb_w": (lambda: synth.barabasi_albert(800, 3, seed=5), COMBINATORIAL, False, 7),
    # tr L^2 is summed in chunks of 8192 values: three diagonal chunks (the
    # last ragged) and several entry chunks
    "ba20000": (lambda: synth.barabasi_albert(20000, 2, seed=8), NORMALIZED, False, None),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("degree", [1, 2])
def test_cv_matches_oracle(name, degree):
    gen, kind, drop, wseed = CASES[name]
    s, d, n = gen()
    w = None if wseed is None else np.random.default_rng(wseed).uniform(0.5, 2.0, s.size)
    lap = build_laplacian(s, d, n, weights=w, kind=kind, drop_isolated=drop)
    g = slaq.build_laplacian(_dev(s), _dev(d), n, weights=None if w is None else _dev(w, torch.float64),
                             kind=slaq.NORMALIZED if kind == NORMALIZED else slaq.COMBINATORIAL,
                             flags=slaq.DROP_ISOLATED if drop else 0)
    nv, steps, seed = 12, 12, 4
    K = slaq.lanczos(g, nv, steps, seed, precision=slaq.FP64)
    t = synth.t_grid(64)
    h, se = (x.cpu().numpy() for x in slaq.trace_heat_cv(K, _dev(t, torch.float64), degree))
    runs = odesc.slq_runs(lap, steps, nv, seed)
    oh, ose = ovar.heat_trace_cv(runs, lap.n, t, degree, lap.norm_bound(), lap.trace,
                                 ovar.frobenius_sq(lap))
    # exp(-t theta) turns the eigensolver's absolute error into t ||L|| eps relative
    rt = np.maximum(RTOL, t * lap.norm_bound() * 1e-14)
    assert np.all(np.abs(h - oh) <= rt * np.abs(oh)), name
    assert np.all(np.abs(se - ose) <= 1e-6 * ose + 1e-9 * lap.n), name


def test_cv_batch_per_graph():
    empty = (np.zeros(0, np.int32), np.zeros(0, np.int32), 4)  # all nodes dropped
    graphs = [synth.barabasi_albert(300, 3, seed=1), synth.sbm([40, 40, 41], 0.3, 0.02, seed=2),
              empty, synth.cycle(17), synth.rmat(11, 8 << 11, seed=4),
              synth.barabasi_albert(9000, 3, seed=7)]  # 2 diagonal chunks of tr L^2
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    nv, steps, seed = 6, 10, 5
    K = slaq.lanczos(gb, nv, steps, seed, precision=slaq.FP64)
    t = synth.t_grid(32)
    h = slaq.trace_heat_cv(K, _dev(t, torch.float64), 2)[0].cpu().numpy()
    assert h.shape == (len(graphs), t.size)
    assert np.all(h[2] == 0.0)
    for gi, (s, d, n) in enumerate(graphs):
        if gi == 2:
            continue
        lap = build_laplacian(s, d, n, drop_isolated=True)
        runs = odesc.slq_runs(lap, steps, nv, seed, graph=gi)
        oh, _ = ovar.heat_trace_cv(runs, lap.n, t, 2, lap.norm_bound(), lap.trace,
                                   ovar.frobenius_sq(lap))
        np.testing.assert_allclose(h[gi], oh, rtol=RTOL)


def test_cv_reduced_forms_and_variance_reduction():
    s, d, n = synth.rmat(14, 16 << 14, seed=6)
    g = slaq.build_laplacian(_dev(s), _dev(d), n, flags=slaq.DROP_ISOLATED)
    t = _dev(np.array([0.01, 0.1, 1.0, 10.0]), torch.float64)
    K64 = slaq.lanczos(g, 32, 15, 2, precision=slaq.FP64)
    h64, se64 = slaq.trace_heat_cv(K64, t, 2)
    plain, plain_se = slaq.trace_heat(K64, t)
    # unbiased: the two estimates agree within their errors; the variance falls
    assert torch.all(torch.abs(h64 - plain) <= 4 * plain_se).item()
    ratio = (plain_se / se64).cpu().numpy()
    assert ratio[0] > 100 and ratio[1] > 10 and ratio[2] > 1.5, ratio
    for prec in (slaq.FP32, slaq.FP32_BF16BASIS):
        h = slaq.trace_heat_cv(slaq.lanczos(g, 32, 15, 2, precision=prec), t, 2)[0]
        assert torch.max(torch.abs(h - h64) / h64).item() < 1e-4, prec
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.trace_heat_cv(K64, t, 3)
    assert ei.value.status == 1


@pytest.mark.parametrize("nv,steps", [(512, 6), (3, 64), (1, 8)])
def test_cv_largest_sizes_and_one_probe(nv, steps):
    """The control variate at the largest probe block and step count the
    library accepts, and with one probe (no standard error: NaN)."""
    s, d, n = synth.barabasi_albert(2000, 4, seed=0)
    lap = build_laplacian(s, d, n)
    g = slaq.build_laplacian(_dev(s), _dev(d), n)
    K = slaq.lanczos(g, nv, steps, 3, precision=slaq.FP64)
    t = synth.t_grid(32)
    h, se = (x.cpu().numpy() for x in slaq.trace_heat_cv(K, _dev(t, torch.float64), 2))
    runs = odesc.slq_runs(lap, steps, nv, 3)
    oh, ose = ovar.heat_trace_cv(runs, lap.n, t, 2, lap.norm_bound(), lap.trace,
                                 ovar.frobenius_sq(lap))
    rt = np.maximum(RTOL, t * lap.norm_bound() * 1e-14)
    assert np.all(np.abs(h - oh) <= rt * np.abs(oh))
    if nv == 1:
        assert np.all(np.isnan(se))
    else:
        assert np.all(np.abs(se - ose) <= 1e-6 * ose + 1e-9 * lap.n)
