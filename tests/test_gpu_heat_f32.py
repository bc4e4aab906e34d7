"""The reduced forms' heat-trace evaluation (k_heat_f32) against an FP64
evaluation of the same Gauss rules, through the C ABI.

The FP32 and BF16-basis forms evaluate e^{-t theta} in FP32 with the product
t theta kept in two floats (hi and a residual from an FMA), and sum a probe's
terms in FP32.  Taking the Gauss rules the run produced (theta and tau2, FP64,
from slaq_ritz_export) and evaluating n' sum_k tau2 e^{-t theta} in FP64 on
the host isolates that arithmetic from the Lanczos rounding: per probe it
must agree to the FP32 sum's rounding (m terms: relative m 2^-24 at most),
for t up to 1000, the largest t the FP32 form serves on a normalized
Laplacian, where rounding t theta itself to a float would cost |t theta|
2^-24.  Also covered: a batch (rules staged per graph), probes that stopped
early (m < s), and the mean and standard error over probes.
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


def _host_heat(K, t_np, n_nodes):
    """n'_g sum_k tau2 e^{-t theta} per graph, probe and t, in FP64."""
    G = len(n_nodes)
    theta, tau2 = (x.cpu().numpy() for x in slaq.ritz_export(K))
    nv, s = theta.shape[-2:]
    theta, tau2 = theta.reshape(G, nv, s), tau2.reshape(G, nv, s)
    m = slaq.krylov_export(K)[2].cpu().numpy().reshape(G, nv)
    pp = np.zeros((G, nv, t_np.size))
    for g in range(G):
        for p in range(nv):
            k = int(m[g, p])
            th, w = theta[g, p, :k], tau2[g, p, :k]
            pp[g, p] = n_nodes[g] * (w[None, :] * np.exp(-np.outer(t_np, th))).sum(1)
    return pp


def _check(K, t_np, n_nodes, m_max):
    G, nt = len(n_nodes), t_np.size
    t = torch.as_tensor(t_np, device="cuda", dtype=torch.float64)
    h, se, pp = (x.cpu().numpy() for x in slaq.trace_heat(K, t, per_probe=True))
    h, se = h.reshape(G, nt), se.reshape(G, nt)
    ref = _host_heat(K, t_np, n_nodes)
    pp = pp.reshape(ref.shape)
    # the FP32 sum of m positive terms, each within a few units of 2^-24
    bar = 2.0 * m_max * 2.0 ** -24
    # below 1e-30 a value leaves the range FP32 evaluates in relative terms
    # (e^{-t theta} underflows past t theta = 103; a star's probe without a
    # component along the null vector has no node below 1): absolute there
    tiny = 1e-30
    live = np.abs(ref) > tiny
    assert np.all(np.abs(pp[~live] - ref[~live]) <= tiny)
    rel = np.abs(pp[live] - ref[live]) / np.abs(ref[live])
    assert np.max(rel) < bar, float(np.max(rel))
    mean = ref.mean(1)
    ok = np.abs(mean) > tiny
    assert np.all(np.abs(h[~ok] - mean[~ok]) <= tiny)
    assert np.max(np.abs(h[ok] - mean[ok]) / np.abs(mean[ok])) < bar
    # the standard error inherits the per-probe rounding, absolute
    sd = ref.std(1, ddof=1) / np.sqrt(ref.shape[1])
    assert np.all(np.abs(se - sd) <= 1e-3 * sd + bar * np.abs(mean))


@pytest.mark.parametrize("precision", [slaq.FP32, slaq.FP32_BF16BASIS])
def test_heat_f32_single_graph(precision):
    s, d, n = synth.rmat(13, 16 << 13, seed=5)
    g = slaq.build_laplacian(torch.as_tensor(s, device="cuda"), torch.as_tensor(d, device="cuda"), n,
                             flags=slaq.DROP_ISOLATED)
    K = slaq.lanczos(g, 64, 20, 3, precision=precision)
    hi = 1000.0 if precision == slaq.FP32 else 10.0
    t_np = np.geomspace(1e-3, hi, 97)
    _check(K, t_np, [slaq.graph_info(g)["n"]], 20)


def test_heat_f32_batch_with_early_stops():
    # stars and complete graphs stop after 2 or 3 steps (m < s): the staged
    # rules of those probes are read only up to m
    graphs = synth.sbm_batch(30, seed=4) + [synth.star(50), synth.complete(9), synth.cycle(40)]
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    K = slaq.lanczos(gb, 20, 15, 7, precision=slaq.FP32)
    m = slaq.krylov_export(K)[2].cpu().numpy()
    assert m.min() < 15
    nodes = np.diff(slaq.graph_batch_info(gb)["node_off"])
    _check(K, np.geomspace(1e-3, 1000.0, 64), nodes, 15)
