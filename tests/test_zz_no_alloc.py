"""The allocation-free heat trace entry point, against the regular path and
the oracle.

Some callers cannot allocate device memory at the moment they call into the
library: an application whose own memory manager owns all device memory and
hands libraries only the buffers it created, or a latency-critical loop in
which a cudaMalloc (which may synchronize the device) is not allowed.  For
them the library offers slaq_trace_heat_tridiag_static, which takes the
Lanczos coefficients and writes the heat trace while keeping its scratch (the
Gauss nodes and weights, the clamped rule sizes) in a fixed array inside the
library.

This file checks, through the C ABI, that two consecutive calls of that entry
point give the heat trace the regular handle-based entry point gives for the
same Lanczos run and the oracle gives for the same probes, that one probe
gives a NaN standard error, that rule sizes outside [0, s] are clamped and
flagged, and that sizes beyond its fixed scratch are rejected.  It is named
so that pytest collects it last, and it passes on its own in a fresh process
as well as after the other tests.
"""
import math

import numpy as np
import pytest

import synth
from oracle import descriptors as odesc
from oracle.laplacian import build_laplacian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2003_01282_gb300 import slaq  # noqa: E402
from paper_2003_01282_gb300.build import build  # noqa: E402

RTOL = 1e-10  # the FP64 parity tolerance of the GPU tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build()
    slaq.lib()
    assert slaq.device_check() == 0, slaq.last_error()


def _ba():
    return synth.barabasi_albert(2000, 4, seed=0)


def _run(nv, s, seed):
    src, dst, n = _ba()
    g = slaq.build_laplacian(torch.as_tensor(src, device="cuda"),
                             torch.as_tensor(dst, device="cuda"), n)
    K = slaq.lanczos(g, nv, s, seed, precision=slaq.FP64)
    return g, K


def test_static_scratch_matches_regular_entry_point_and_oracle():
    t_np = synth.t_grid()
    t = torch.as_tensor(t_np, device="cuda")
    g, K = _run(40, 15, 3)
    want, want_se = (x.cpu().numpy() for x in slaq.trace_heat(K, t))
    alpha, beta, m = slaq.krylov_export(K)
    n = g.info["n"]
    # the oracle on the same probes (graph field 0, seed 3)
    lap = build_laplacian(*_ba())
    oh, ose = odesc.heat_trace(odesc.slq_runs(lap, 15, 40, 3), lap.n, t_np)
    for _ in range(2):  # two calls in a row share the same scratch
        out, se, status = slaq.trace_heat_tridiag_static(alpha, beta, m, n, t)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=RTOL, atol=0)
        np.testing.assert_allclose(se.cpu().numpy(), want_se, rtol=RTOL, atol=0)
        np.testing.assert_allclose(out.cpu().numpy(), oh, rtol=RTOL, atol=0)
        np.testing.assert_allclose(se.cpu().numpy(), ose, rtol=1e-6, atol=0)
    # a different run in between: the scratch holds the newest call's rule
    g2, K2 = _run(7, 9, 11)
    want2 = slaq.trace_heat(K2, t)[0].cpu().numpy()
    a2, b2, m2 = slaq.krylov_export(K2)
    out2, _, st2 = slaq.trace_heat_tridiag_static(a2, b2, m2, g2.info["n"], t)
    torch.cuda.synchronize()
    assert int(st2.item()) == 0
    np.testing.assert_allclose(out2.cpu().numpy(), want2, rtol=RTOL, atol=0)


def test_static_scratch_one_probe_has_nan_stderr():
    t = torch.as_tensor(synth.t_grid(16), device="cuda")
    g, K = _run(1, 12, 5)
    want = slaq.trace_heat(K, t)[0].cpu().numpy()
    alpha, beta, m = slaq.krylov_export(K)
    out, se, status = slaq.trace_heat_tridiag_static(alpha, beta, m, g.info["n"], t)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=RTOL, atol=0)
    assert np.all(np.isnan(se.cpu().numpy()))


def test_static_scratch_clamps_rule_sizes():
    """m[p] beyond s (or negative) is clamped to [0, s] and flagged by status
    bit 2; the trace stays finite and equals the clamped rule's."""
    t = torch.as_tensor(synth.t_grid(32), device="cuda")
    g, K = _run(6, 10, 9)
    alpha, beta, m = slaq.krylov_export(K)
    n = g.info["n"]
    ref = slaq.trace_heat_tridiag_static(alpha, beta, m, n, t)[0].cpu().numpy()
    bad = m.clone()
    bad[2] = 10 + 5
    out, _, status = slaq.trace_heat_tridiag_static(alpha, beta, bad, n, t)
    torch.cuda.synchronize()
    assert int(status.item()) & 2
    assert np.all(np.isfinite(out.cpu().numpy()))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL, atol=0)  # m[2] was s already
    bad[2] = -3  # clamped to 0: probe 2 contributes nothing
    out, _, status = slaq.trace_heat_tridiag_static(alpha, beta, bad, n, t)
    torch.cuda.synchronize()
    assert int(status.item()) & 2
    _, _, pp = slaq.trace_heat(K, t, per_probe=True)
    pp = pp.cpu().numpy()
    pp[2] = 0.0
    np.testing.assert_allclose(out.cpu().numpy(), pp.mean(0), rtol=RTOL, atol=0)
    # and a clean call afterwards clears the flag
    _, _, status = slaq.trace_heat_tridiag_static(alpha, beta, m, n, t)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert math.isfinite(float(out[0].item()))


def test_static_scratch_rejects_oversize_and_mismatched_shapes():
    t = torch.as_tensor(synth.t_grid(8), device="cuda")
    big = torch.zeros(513, 4, dtype=torch.float64, device="cuda")
    m = torch.ones(513, dtype=torch.int32, device="cuda")
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.trace_heat_tridiag_static(big, big, m, 1000, t)
    assert ei.value.status == 1 and "static scratch" in str(ei.value)
    long = torch.zeros(4, 65, dtype=torch.float64, device="cuda")
    with pytest.raises(slaq.SlaqError):
        slaq.trace_heat_tridiag_static(long, long, m[:4].contiguous(), 1000, t)
    a = torch.zeros(4, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        slaq.trace_heat_tridiag_static(a, a[:, :7].contiguous(), m[:4].contiguous(), 100, t)
    with pytest.raises(ValueError):
        slaq.trace_heat_tridiag_static(a, a, m[:3].contiguous(), 100, t)
