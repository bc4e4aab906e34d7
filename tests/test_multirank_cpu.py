"""Probe sharding over processes on CPU (gloo, world size 2).

The path shards probes (Sec. 3.1, Eq. trace: the probes are independent):
rank r runs a range of the probe generator's probes of ONE seed
(slaq_lanczos_probes on a GPU), the ranks all-gather their per-probe values
and pool them with slaq_pool_probes_host.  The pooled mean and standard
error must equal those of one process over all the probes.  Without a GPU
the per-probe values come from the oracle for each rank's probe range; the
exchange and the pooling are the ones the GPU path uses.  The job's step time
is the slowest rank's.
"""
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2
NV, STEPS, SEED = 7, 8, 4   # 7 probes: an uneven split (4 + 3)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import synth
    from oracle.laplacian import build_laplacian
    s, d, n = synth.barabasi_albert(200, 3, seed=0)
    return build_laplacian(s, d, n), synth.t_grid(16)


def _values(lap, t, probes):
    """Per-probe [heat | wave re | wave im | vnge] rows for the given probes."""
    from oracle import descriptors as od
    runs = od.slq_runs(lap, STEPS, NV, SEED, probes=probes)
    n = lap.n
    heat = od.per_probe(runs, od.heat_f(t)) * n
    wr = od.per_probe(runs, od.wave_re_f(t)) * n
    wi = od.per_probe(runs, od.wave_im_f(t)) * n
    vn = od.per_probe(runs, od.vnge_f(lap.trace))[:, None] * n
    return np.concatenate([heat, wr, wi, vn], axis=1)


def _worker(rank, port, queue):
    import os
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as tdist
    tdist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import bench
        from paper_2003_01282_gb300 import shard
        lap, t = _problem()
        p0, nv = shard.probe_range(rank, WORLD, NV)
        local = torch.as_tensor(_values(lap, t, range(p0, p0 + nv)))
        full = shard.gather_probe_values(local, NV, tdist)
        mean, se = shard.pool(full)
        ms = bench.max_over_ranks(10.0 + rank, torch.device("cpu"), tdist)
        queue.put((rank, (p0, nv), mean, se, ms))
    finally:
        tdist.destroy_process_group()


def test_probe_range_split():
    from paper_2003_01282_gb300 import shard
    assert [shard.probe_range(r, 2, 7) for r in range(2)] == [(0, 4), (4, 3)]
    assert [shard.probe_range(r, 3, 100) for r in range(3)] == [(0, 34), (34, 33), (67, 33)]
    with pytest.raises(ValueError):
        shard.probe_range(2, 2, 7)


def test_pool_matches_numpy_and_single_probe():
    from paper_2003_01282_gb300 import shard
    rng = np.random.default_rng(1)
    v = rng.normal(3.0, 2.0, size=(13, 5))
    mean, se = shard.pool(v)
    np.testing.assert_allclose(mean, v.mean(0), rtol=1e-14)
    np.testing.assert_allclose(se, v.std(0, ddof=1) / np.sqrt(13), rtol=1e-13)
    mean, se = shard.pool(v[:1])
    np.testing.assert_array_equal(mean, v[0])
    assert np.all(np.isnan(se))


def test_probe_sharding_two_ranks():
    import bench
    from oracle import descriptors as od
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, queue)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(WORLD):
        rank, rng_, mean, se, ms = queue.get(timeout=180)
        out[rank] = (rng_, mean, se, ms)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == (0, 4) and out[1][0] == (4, 3)
    # the oracle's estimate over all NV probes of the seed, in one process
    lap, t = _problem()
    runs = od.slq_runs(lap, STEPS, NV, SEED)
    h, hse = od.heat_trace(runs, lap.n, t)
    (wr, wrse), (wi, wise) = od.wave_trace(runs, lap.n, t)
    v, vse = od.vnge(runs, lap.n, lap.trace)
    want = np.concatenate([h, wr, wi, [v]])
    want_se = np.concatenate([hse, wrse, wise, [vse]])
    for rank in range(WORLD):
        _, mean, se, ms = out[rank]
        np.testing.assert_allclose(mean, want, rtol=1e-12, atol=1e-12 * lap.n)
        np.testing.assert_allclose(se, want_se, rtol=1e-9, atol=1e-12 * lap.n)
        assert ms == 11.0
    assert bench.whole_job_value(2, 1000.0, 10.0) == 2 * 1000.0 / 0.01
