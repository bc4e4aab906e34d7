"""The orthogonality monitor (slaq_krylov_monitor) through the C ABI.

max |Q^T Q - I| of the stored Lanczos basis, from the Gram entries the run
measures, and the smallest beta: the FP64 form keeps the basis orthogonal to
working precision (the oracle's basis passes 1e-12 in the CPU pins), the
FP32 and BF16 forms to their storage precision; min beta equals the smallest
exported beta; a breakdown graph reports its truncated rules' betas.
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


def _g(edges, **kw):
    s, d, n = edges
    return slaq.build_laplacian(torch.as_tensor(s, device="cuda"), torch.as_tensor(d, device="cuda"),
                                n, **kw)


@pytest.mark.parametrize("precision,bar", [(slaq.FP64, 1e-12), (slaq.FP32, 1e-5),
                                           (slaq.FP32_BF16BASIS, 3e-2)])
def test_monitor_orthogonality_and_min_beta(precision, bar):
    g = _g(synth.barabasi_albert(2000, 4, seed=0))
    K = slaq.lanczos(g, 16, 15, 3, precision=precision)
    mon = slaq.krylov_monitor(K)
    assert 0.0 < mon["ortho"] < bar, mon
    _, beta, m = slaq.krylov_export(K)
    beta, m = beta.cpu().numpy(), m.cpu().numpy()
    want = min(beta[p, :m[p] - 1].min() for p in range(16))
    assert mon["min_beta"] == want
    # partial reorthogonalization: semi-orthogonal (sqrt(eps) bar) by design
    if precision != slaq.FP32_BF16BASIS:
        Kp = slaq.lanczos(g, 16, 15, 3, precision=precision, reorth_passes=slaq.REORTH_PARTIAL)
        eps = 2.0 ** -53 if precision == slaq.FP64 else 2.0 ** -24
        assert slaq.krylov_monitor(Kp)["ortho"] < 10 * np.sqrt(eps)


def test_monitor_breakdown_graph_and_batch():
    # K_9: every probe's Krylov space closes after at most two vectors (one
    # beta); a probe of one sign throughout is the null vector itself (m = 1)
    g = _g(synth.complete(9))
    K = slaq.lanczos(g, 6, 8, 1, precision=slaq.FP64)
    mon = slaq.krylov_monitor(K)
    _, beta, m = slaq.krylov_export(K)
    m, beta = m.cpu().numpy(), beta.cpu().numpy()
    assert np.all((m >= 1) & (m <= 2)) and np.any(m == 2)
    assert mon["min_beta"] == beta[m == 2, 0].min()
    assert mon["ortho"] < 1e-12
    # a batch: the worst over its graphs
    graphs = synth.sbm_batch(40, seed=3)
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    Kb = slaq.lanczos(gb, 8, 10, 2, precision=slaq.FP32)
    assert slaq.krylov_monitor(Kb)["ortho"] < 1e-5
