"""Probe ranges (slaq_lanczos_probes) and their pooling, through the C ABI.

Sec. 3.1 / Eq. trace: the Hutchinson estimate averages independent probes, so
a run over probes 0..nv-1 can be split into ranges of the probe generator
(one per GPU, or chunks that fit memory).  Checks:
* each range's per-probe values (heat, wave, VNGE) equal the matching rows of
  the run over all probes (FP64, relative 1e-12: only the dot products'
  summation order differs) and the oracle's for those probe indices (1e-10);
* the ranges' per-probe values pooled by slaq_pool_probes_host give the
  single run's means and standard errors;
* slaq_trace_wave_per_probe averages to slaq_trace_wave;
* a rerun keeps the range; ranges beyond the 16-bit probe field are refused.
"""
import numpy as np
import pytest

import synth
from oracle import descriptors as odesc
from oracle.laplacian import build_laplacian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2003_01282_gb300 import shard, slaq  # noqa: E402
from paper_2003_01282_gb300.build import build  # noqa: E402

NV, S, SEED = 24, 12, 7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build()
    slaq.lib()


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _graph():
    s, d, n = synth.rmat(12, 16 << 12, seed=3)
    return (s, d, n), slaq.build_laplacian(torch.as_tensor(s, device="cuda"),
                                           torch.as_tensor(d, device="cuda"), n,
                                           flags=slaq.DROP_ISOLATED)


def _values(K, t):
    heat = slaq.trace_heat(K, t, per_probe=True)[2]
    re, im = slaq.trace_wave_per_probe(K, t)
    vn = slaq.trace_vnge(K, per_probe=True)[2]
    return torch.cat([heat, re, im, vn[:, None]], dim=1).cpu().numpy()


@pytest.mark.parametrize("precision", [slaq.FP64, slaq.FP32])
def test_ranges_equal_rows_of_one_run_and_pool_to_it(precision):
    (s, d, n), g = _graph()
    t_np = synth.t_grid(64)
    t = torch.as_tensor(t_np, device="cuda")
    K = slaq.lanczos(g, NV, S, SEED, precision=precision)
    whole = _values(K, t)
    h, hse = (x.cpu().numpy() for x in slaq.trace_heat(K, t))
    (wr, wrse), (wi, wise) = slaq.trace_wave(K, t)
    v, vse = (x.cpu().numpy() for x in slaq.trace_vnge(K))
    # slaq_trace_wave_per_probe averages to slaq_trace_wave
    np.testing.assert_allclose(whole[:, 64:128].mean(0), wr.cpu().numpy(), rtol=1e-13,
                               atol=1e-13 * g.info["n"])
    parts = []
    for p0, nv in ((0, 10), (10, 14)):
        Kr = slaq.lanczos_probes(g, nv, p0, S, SEED, precision=precision)
        vals = _values(Kr, t)
        tol = 1e-12 if precision == slaq.FP64 else 1e-5
        np.testing.assert_allclose(vals, whole[p0:p0 + nv], rtol=tol, atol=tol * g.info["n"])
        parts.append(vals)
    mean, se = shard.pool(np.concatenate(parts))
    want = np.concatenate([h, wr.cpu().numpy(), wi.cpu().numpy(), v])
    want_se = np.concatenate([hse, wrse.cpu().numpy(), wise.cpu().numpy(), vse])
    tol = 1e-12 if precision == slaq.FP64 else 1e-5
    np.testing.assert_allclose(mean, want, rtol=tol, atol=tol * g.info["n"])
    np.testing.assert_allclose(se, want_se, rtol=1e-6 if precision == slaq.FP64 else 1e-2,
                               atol=tol * g.info["n"])
    if precision == slaq.FP64:
        # the second range against the oracle at those probe indices
        lap = build_laplacian(s, d, n, drop_isolated=True)
        runs = odesc.slq_runs(lap, S, NV, SEED, probes=range(10, 24))
        oh = odesc.per_probe(runs, odesc.heat_f(t_np)) * lap.n
        assert _rel(parts[1][:, :64], oh) < 1e-10


def test_rerun_keeps_the_range_and_limits():
    (_, _, _), g = _graph()
    t = torch.as_tensor(synth.t_grid(16), device="cuda")
    K = slaq.lanczos_probes(g, 5, 300, S, SEED, precision=slaq.FP64)
    slaq.lanczos_rerun(K, SEED + 1)
    a = slaq.trace_heat(K, t, per_probe=True)[2].cpu().numpy()
    Kf = slaq.lanczos_probes(g, 5, 300, S, SEED + 1, precision=slaq.FP64)
    b = slaq.trace_heat(Kf, t, per_probe=True)[2].cpu().numpy()
    np.testing.assert_array_equal(a, b)
    # a reused handle going back to probe 0 starts from probe 0 again
    slaq.lanczos(g, 5, S, SEED + 1, precision=slaq.FP64, reuse=Kf)
    c = slaq.trace_heat(Kf, t, per_probe=True)[2].cpu().numpy()
    K0 = slaq.lanczos_probes(g, 5, 0, S, SEED + 1, precision=slaq.FP64)
    np.testing.assert_array_equal(c, slaq.trace_heat(K0, t, per_probe=True)[2].cpu().numpy())
    for p0, nv in ((-1, 4), (65533, 4), (65536, 1)):
        with pytest.raises(slaq.SlaqError) as ei:
            slaq.lanczos_probes(g, nv, p0, S, SEED)
        assert ei.value.status == 1
    slaq.lanczos_probes(g, 4, 65532, S, SEED)  # the last four probes of the field


@pytest.mark.parametrize("precision", [slaq.FP64, slaq.FP32, slaq.FP32_BF16BASIS])
def test_host_pool_reproduces_device_moments_bit_for_bit(precision):
    """slaq_pool_probes_host over one run's per-probe values gives the
    device's mean and standard error exactly: the same Welford updates per
    probe group and Chan merge in group order as the quadrature kernels
    (heat through k_trace_t for FP64 and k_heat_f32 for the reduced forms)."""
    _, g = _graph()
    K = slaq.lanczos(g, 37, S, SEED, precision=precision)
    t_np = synth.t_grid(40)
    if precision == slaq.FP32_BF16BASIS:
        t_np = t_np[t_np * 2.0 <= 20.0]
    t = torch.as_tensor(t_np, device="cuda", dtype=torch.float64)
    h, hse, pp = slaq.trace_heat(K, t, per_probe=True)
    mean, se = slaq.pool_probes_host(pp.cpu().numpy())
    np.testing.assert_array_equal(mean, h.cpu().numpy())
    np.testing.assert_array_equal(se, hse.cpu().numpy())
