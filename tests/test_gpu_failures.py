"""Out-of-memory paths, walked one allocation at a time (host-side injection).

slaq_debug_fail_alloc(n) makes the n-th library allocation after the call
fail as an out-of-memory device would.  For each entry point below, the test
arms the hook for n = 1, 2, ... until the call succeeds: every failing call
must return SLAQ_ENOMEM, release what it allocated (slaq_debug_live_allocs
back to its value before the call), and leave every handle it was given
destroyable; a Krylov handle whose run failed must refuse to be read
(SLAQ_EINVAL) and must run again correctly.  Nothing here faults, traps or
hangs the GPU: the failure is a host-side return code, and no kernel is
launched after it.
"""
import gc

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2003_01282_gb300 import slaq  # noqa: E402
from paper_2003_01282_gb300.build import build  # noqa: E402

ENOMEM, EINVAL = 2, 1
MAX_STEPS = 400


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build()
    slaq.lib()
    yield
    slaq.debug_fail_alloc(0)


def _dev(a):
    return torch.as_tensor(a, device="cuda")


class _NoCycleCollection:
    """Collects garbage once, then keeps Python's cycle collector off: handles
    held only by reference cycles (an earlier test's exception traceback)
    would otherwise be freed in the middle of a walk and move the count."""

    def __enter__(self):
        gc.collect()
        gc.disable()

    def __exit__(self, *exc):
        gc.enable()


def _walk(call, cleanup=lambda: None):
    """Runs call() with the n-th allocation failing, n = 1, 2, ..., until it
    succeeds; returns (number of failures seen, the successful result)."""
    with _NoCycleCollection():
        torch.cuda.synchronize()
        base = slaq.debug_live_allocs()
        for n in range(1, MAX_STEPS):
            slaq.debug_fail_alloc(n)
            try:
                out = call()
            except slaq.SlaqError as e:
                slaq.debug_fail_alloc(0)
                assert e.status == ENOMEM, (n, str(e))
                cleanup()
                torch.cuda.synchronize()
                assert slaq.debug_live_allocs() == base, (n, "leak after a failed call")
                continue
            slaq.debug_fail_alloc(0)
            return n - 1, out
    raise AssertionError("the call never succeeded")


def _graph_edges(n=600):
    return synth.barabasi_albert(n, 4, seed=5)


def test_build_laplacian_every_allocation():
    s, d, n = _graph_edges()
    src, dst = _dev(s), _dev(d)
    fails, g = _walk(lambda: slaq.build_laplacian(src, dst, n, flags=slaq.DROP_ISOLATED))
    assert fails >= 20  # validation, sort, CSR, execution copy, schedules
    ref = slaq.build_laplacian(src, dst, n, flags=slaq.DROP_ISOLATED)
    a, b = slaq.graph_export(g), slaq.graph_export(ref)
    for k in ("rowptr", "colidx", "vals", "diag", "old_id"):
        assert torch.equal(a[k], b[k]), k
    g.close()
    ref.close()
    # a weighted batch (more arrays, the per-graph tables)
    graphs = [synth.barabasi_albert(40 + 5 * i, 3, seed=i) for i in range(6)]
    w = [np.random.default_rng(i).uniform(0.5, 2, x[0].size) for i, x in enumerate(graphs)]
    fails, gb = _walk(lambda: slaq.build_laplacian_batch(graphs, weights=w, kind=slaq.COMBINATORIAL))
    assert fails >= 20
    gb.close()


@pytest.mark.parametrize("precision,reorth", [(slaq.FP64, 1), (slaq.FP32, 1), (slaq.FP32_BF16BASIS, 1),
                                              (slaq.FP32, slaq.REORTH_PARTIAL), (slaq.FP64, 2)])
def test_lanczos_fresh_handle_every_allocation(precision, reorth):
    s, d, n = _graph_edges()
    g = slaq.build_laplacian(_dev(s), _dev(d), n)
    t = _dev(synth.t_grid(32)[:24])  # t <= 10: every form serves it
    fails, K = _walk(lambda: slaq.lanczos(g, 12, 10, 3, precision=precision, reorth_passes=reorth))
    assert fails >= 10
    want = slaq.trace_heat(slaq.lanczos(g, 12, 10, 3, precision=precision, reorth_passes=reorth), t)[0]
    assert torch.equal(slaq.trace_heat(K, t)[0], want)


def test_reused_handle_failing_to_grow_stays_usable():
    """A handle built on a small graph, grown for a larger one with the n-th
    allocation failing: the call fails, the handle refuses to be read or
    replayed, and the next run on it (no failure) equals a fresh handle's."""
    s, d, n = _graph_edges(300)
    small = slaq.build_laplacian(_dev(s), _dev(d), n)
    s2, d2, n2 = synth.rmat(13, 16 << 13, seed=3)   # split rows: the heavy-row buffers grow too
    big = slaq.build_laplacian(_dev(s2), _dev(d2), n2, flags=slaq.DROP_ISOLATED)
    t = _dev(synth.t_grid(16))
    for precision in (slaq.FP32, slaq.FP64):
        want = slaq.trace_heat(slaq.lanczos(big, 20, 8, 5, precision=precision), t)[0]
        failures = 0
        for nth in range(1, MAX_STEPS):
            K = slaq.lanczos(small, 20, 8, 5, precision=precision)
            gc.collect()
            torch.cuda.synchronize()
            base = slaq.debug_live_allocs()
            slaq.debug_fail_alloc(nth)
            try:
                slaq.lanczos(big, 20, 8, 5, precision=precision, reuse=K)
                ok = True
            except slaq.SlaqError as e:
                ok = False
                assert e.status == ENOMEM
            slaq.debug_fail_alloc(0)
            if ok:
                assert torch.equal(slaq.trace_heat(K, t)[0], want)
                K.close()
                break
            failures += 1
            with pytest.raises(slaq.SlaqError) as ei:
                slaq.trace_heat(K, t)
            assert ei.value.status == EINVAL
            with pytest.raises(slaq.SlaqError) as ei:
                slaq.lanczos_rerun(K, 9)
            assert ei.value.status == EINVAL
            torch.cuda.synchronize()
            assert slaq.debug_live_allocs() <= base + 1  # a grown buffer may replace a freed one
            slaq.lanczos(big, 20, 8, 5, precision=precision, reuse=K)  # runs again, no failure
            assert torch.equal(slaq.trace_heat(K, t)[0], want)
            K.close()
        assert failures >= 5


def test_batched_rayleigh_ritz_and_host_entry_point():
    # >= 4096 problems in a reduced form: the Rayleigh-Ritz step's scratch
    graphs = synth.sbm_batch(220, seed=7)
    gb = slaq.build_laplacian_batch(graphs, flags=slaq.DROP_ISOLATED)
    fails, K = _walk(lambda: slaq.lanczos(gb, 20, 10, 2, precision=slaq.FP32))
    assert fails >= 10
    t = _dev(synth.t_grid(16))
    want = slaq.trace_heat(slaq.lanczos(gb, 20, 10, 2, precision=slaq.FP32), t)[0]
    assert torch.equal(slaq.trace_heat(K, t)[0], want)
    # slaq_lanczos_batched over separate handles (the concatenation)
    parts = [slaq.build_laplacian(_dev(a), _dev(b), nn) for a, b, nn in graphs[:5]]
    fails, Kb = _walk(lambda: slaq.lanczos_batched(parts, 8, 6, 1, precision=slaq.FP64))
    assert fails >= 10
    # the host-memory entry point (with no workspace kept from an earlier
    # call; the successful call keeps its own, which the second call reuses)
    s, d, n = _graph_edges()
    tn = synth.t_grid(8)
    slaq.release_cached()
    base = slaq.debug_live_allocs()
    fails, out = _walk(lambda: slaq.descriptors_host(s, d, n, tn, nv=6, s=8, seed=1))
    assert fails >= 10
    kept = slaq.debug_live_allocs()
    assert kept > base
    ref = slaq.descriptors_host(s, d, n, tn, nv=6, s=8, seed=1)
    np.testing.assert_array_equal(out["heat"], ref["heat"])
    assert slaq.debug_live_allocs() == kept
    # a call failing before it reaches the kept workspace leaves it alone
    slaq.debug_fail_alloc(1)
    with pytest.raises(slaq.SlaqError):
        slaq.descriptors_host(s, d, n, tn, nv=6, s=8, seed=1)
    slaq.debug_fail_alloc(0)
    torch.cuda.synchronize()
    assert slaq.debug_live_allocs() == kept
    slaq.release_cached()
    assert slaq.debug_live_allocs() == base
