"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path shards probes: every rank runs the same graph with its own probe
seed and the per-rank estimates are averaged with one all-reduce; the job's
step time is the slowest rank's.  Here the per-rank estimates come from the
oracle (no GPU), and the pooled result must equal the oracle's estimate over
the union of both ranks' probes.
"""
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import synth
    from oracle.laplacian import build_laplacian
    s, d, n = synth.barabasi_albert(200, 3, seed=0)
    return build_laplacian(s, d, n), synth.t_grid(16)


def _estimate(lap, t, seed):
    from oracle import descriptors as od
    runs = od.slq_runs(lap, 8, 4, seed)
    h, _ = od.heat_trace(runs, lap.n, t)
    v, _ = od.vnge(runs, lap.n, lap.trace)
    return runs, np.concatenate([h, [v]])


def _worker(rank, port, queue):
    import os
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as tdist
    tdist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import bench
        lap, t = _problem()
        _, est = _estimate(lap, t, bench.rank_seed(rank))
        desc = torch.tensor(est)
        bench.average_over_ranks(desc, WORLD, tdist)
        ms = bench.max_over_ranks(10.0 + rank, torch.device("cpu"), tdist)
        queue.put((rank, desc.numpy(), ms))
    finally:
        tdist.destroy_process_group()


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
        rank, desc, ms = queue.get(timeout=120)
        out[rank] = (desc, ms)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert bench.rank_seed(0) != bench.rank_seed(1)
    lap, t = _problem()
    runs0, e0 = _estimate(lap, t, bench.rank_seed(0))
    runs1, e1 = _estimate(lap, t, bench.rank_seed(1))
    # the pooled estimate over both ranks' probes, computed in one place
    h, _ = od.heat_trace(runs0 + runs1, lap.n, t)
    v, _ = od.vnge(runs0 + runs1, lap.n, lap.trace)
    pooled = np.concatenate([h, [v]])
    for rank in range(WORLD):
        desc, ms = out[rank]
        np.testing.assert_allclose(desc, (e0 + e1) / 2, rtol=1e-14)
        np.testing.assert_allclose(desc, pooled, rtol=1e-12)
        assert ms == 11.0
    assert bench.whole_job_value(2, 1000.0, 10.0) == 2 * 1000.0 / 0.01
