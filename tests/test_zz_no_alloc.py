"""The allocation-free heat trace entry point, against the regular path.

Some callers cannot allocate device memory at the moment they call into the
library: code that records work into a CUDA graph, where allocation calls
are not allowed, or applications whose own memory manager owns all device
memory.  For them the library offers slaq_trace_heat_tridiag_static, which
takes the Lanczos coefficients and writes the heat trace while keeping its
scratch (the Gauss nodes and weights) in a fixed array inside the library.

This file checks, through the C ABI, that two consecutive calls of that
entry point give the heat trace the regular handle-based entry point gives
for the same Lanczos run, and that sizes beyond its fixed scratch are
rejected.  It is named so that pytest collects it last, and it passes on its
own in a fresh process as well as after the other tests.
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

RTOL = 1e-10  # the FP64 parity tolerance of the GPU tests


def _run(nv, s, seed):
    src, dst, n = synth.barabasi_albert(2000, 4, seed=0)
    g = slaq.build_laplacian(torch.as_tensor(src, device="cuda"),
                             torch.as_tensor(dst, device="cuda"), n)
    K = slaq.lanczos(g, nv, s, seed, precision=slaq.FP64)
    return g, K


def test_static_scratch_matches_regular_entry_point():
    build()
    slaq.lib()
    assert slaq.device_check() == 0, slaq.last_error()
    t = torch.as_tensor(synth.t_grid(), device="cuda")
    g, K = _run(40, 15, 3)
    want, want_se = (x.cpu().numpy() for x in slaq.trace_heat(K, t))
    alpha, beta, m = slaq.krylov_export(K)
    n = g.info["n"]
    for _ in range(2):  # two calls in a row share the same scratch
        out, se, status = slaq.trace_heat_tridiag_static(alpha, beta, m, n, t)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=RTOL, atol=0)
        np.testing.assert_allclose(se.cpu().numpy(), want_se, rtol=RTOL, atol=0)
    # a different run in between: the scratch holds the newest call's rule
    g2, K2 = _run(7, 9, 11)
    want2 = slaq.trace_heat(K2, t)[0].cpu().numpy()
    a2, b2, m2 = slaq.krylov_export(K2)
    out2, _, st2 = slaq.trace_heat_tridiag_static(a2, b2, m2, g2.info["n"], t)
    torch.cuda.synchronize()
    assert int(st2.item()) == 0
    np.testing.assert_allclose(out2.cpu().numpy(), want2, rtol=RTOL, atol=0)


def test_static_scratch_rejects_oversize():
    build()
    t = torch.as_tensor(synth.t_grid(8), device="cuda")
    big = torch.zeros(513, 4, dtype=torch.float64, device="cuda")
    m = torch.ones(513, dtype=torch.int32, device="cuda")
    with pytest.raises(slaq.SlaqError) as ei:
        slaq.trace_heat_tridiag_static(big, big, m, 1000, t)
    assert ei.value.status == 1 and "static scratch" in str(ei.value)
    long = torch.zeros(4, 65, dtype=torch.float64, device="cuda")
    with pytest.raises(slaq.SlaqError):
        slaq.trace_heat_tridiag_static(long, long, m[:4].contiguous(), 1000, t)
