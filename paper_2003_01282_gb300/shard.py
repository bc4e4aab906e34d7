"""Probe sharding across processes (one per GPU): host logic only.

The Hutchinson estimate of Eq. trace averages independent probes, so a run
over nv probes splits into ranges of the probe generator
(slaq_lanczos_probes).  Rank r runs probes [probe0_r, probe0_r + nv_r) of the
same seed; the ranks exchange their per-probe values (one all-gather of
[nv_r, len] FP64 rows, a few hundred KB) and pool them with
slaq_pool_probes_host.  The pooled mean AND standard error are those of one
run over all the probes (up to the per-probe values' rounding order), which
averaging the ranks' means could not give for the standard error.

torch.distributed carries the exchange (NCCL between GPUs, gloo on CPU);
every computation stays in libslaq.
"""
from __future__ import annotations

import numpy as np

from . import slaq


def probe_range(rank: int, world: int, nv_total: int) -> tuple[int, int]:
    """(probe0, nv) of rank `rank` when nv_total probes split over `world`
    ranks as evenly as possible (the first nv_total % world ranks get one
    more)."""
    if world < 1 or not 0 <= rank < world or nv_total < world:
        raise ValueError("need 0 <= rank < world <= nv_total")
    base, rem = divmod(nv_total, world)
    return rank * base + min(rank, rem), base + (1 if rank < rem else 0)


def gather_probe_values(local, nv_total: int, tdist, group=None):
    """All-gather every rank's per-probe rows ([nv_r, len], this rank's probe
    range) into the [nv_total, len] array in probe order, on every rank.
    `local` is a torch tensor (CUDA for NCCL, CPU for gloo)."""
    import torch
    world = tdist.get_world_size(group)
    rows = [probe_range(r, world, nv_total)[1] for r in range(world)]
    width = int(local.shape[1])
    pad = torch.zeros((max(rows), width), dtype=torch.float64, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    tdist.all_gather(parts, pad, group=group)
    full = torch.cat([p[:n] for p, n in zip(parts, rows)])
    return full.cpu().numpy()


def pool(values) -> tuple[np.ndarray, np.ndarray]:
    """(mean, stderr) over the rows of [nprobe, len] per-probe values."""
    return slaq.pool_probes_host(np.asarray(values, dtype=np.float64))
