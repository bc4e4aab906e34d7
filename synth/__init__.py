"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This module only makes inputs: undirected edge lists (as two int32 arrays
``src``, ``dst``) and the log-spaced time grid.  It holds none of the
method's arithmetic (no Laplacian, no probes, no Lanczos, no quadrature):
both the CUDA path and the CPU oracle receive exactly these arrays.

Generators
----------
* closed-form graphs: complete K_n, cycle C_n, path P_n, star S_n,
  complete bipartite K_{a,b}, disjoint unions (for the spectral pins);
* Barabasi-Albert preferential attachment (the small single-graph workload);
* R-MAT (Chakrabarti et al. 2004) with quadrant probabilities a, b, c, d,
  sampled in rounds until the requested number of unique undirected
  non-loop pairs exists, then truncated in sampling order (stand-in for the
  paper's SNAP / ClueWeb graphs, Tab. 2 and Tab. 5); ``rmat_torch`` draws the
  same distribution with torch's generator on any device, for the
  web-scale sizes numpy takes minutes to sample;
* stochastic block model batches (stand-in for the graph-classification
  collections of Tab. 3);
* edge rewiring of a fraction of edges (graph pairs for distances).

Every generator is a pure function of its arguments and seed (numpy PCG64;
torch's Philox generator for ``rmat_torch``, whose draws depend on the device
and the torch build).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "t_grid", "complete", "cycle", "path", "star", "complete_bipartite",
    "disjoint_union", "barabasi_albert", "rmat", "sbm", "sbm_batch", "rewire",
    "erdos_renyi", "read_edge_file", "rmat_torch",
]


def _pack(edges) -> tuple[np.ndarray, np.ndarray]:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    return e[:, 0].astype(np.int32), e[:, 1].astype(np.int32)


def t_grid(nt: int = 256, lo: float = -2.0, hi: float = 2.0) -> np.ndarray:
    """Log-spaced NetLSD time grid t_k = 10^(lo + (hi-lo) k/(nt-1)), FP64.

    The paper samples t on a logarithmic grid (Sec. 2.2) without fixing it;
    [1e-2, 1e2] with 256 points is the NetLSD default grid.
    """
    if nt == 1:
        return np.array([10.0 ** lo])
    return np.logspace(lo, hi, nt, dtype=np.float64)


# ----------------------------------------------------------------- closed forms
def complete(n: int):
    i, j = np.triu_indices(n, 1)
    return i.astype(np.int32), j.astype(np.int32), n


def cycle(n: int):
    i = np.arange(n)
    return i.astype(np.int32), ((i + 1) % n).astype(np.int32), n


def path(n: int):
    i = np.arange(n - 1)
    return i.astype(np.int32), (i + 1).astype(np.int32), n


def star(n: int):
    """Star on n nodes: centre 0 joined to 1..n-1."""
    j = np.arange(1, n)
    return np.zeros(n - 1, np.int32), j.astype(np.int32), n


def complete_bipartite(a: int, b: int):
    i, j = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return i.ravel().astype(np.int32), j.ravel().astype(np.int32), a + b


def disjoint_union(*graphs, extra_isolated: int = 0):
    """Union of (src, dst, n) triples with ids shifted; optional isolated tail."""
    srcs, dsts, off = [], [], 0
    for s, d, n in graphs:
        srcs.append(np.asarray(s, np.int64) + off)
        dsts.append(np.asarray(d, np.int64) + off)
        off += n
    return (np.concatenate(srcs).astype(np.int32),
            np.concatenate(dsts).astype(np.int32), off + extra_isolated)


def read_edge_file(path_: str):
    """Read a whitespace edge list with '%' comment lines and '% n_nodes N'."""
    n = None
    rows = []
    with open(path_) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            if line.startswith("%"):
                parts = line[1:].split()
                if len(parts) == 2 and parts[0] == "n_nodes":
                    n = int(parts[1])
                continue
            a, b = line.split()[:2]
            rows.append((int(a), int(b)))
    s, d = _pack(rows)
    if n is None:
        n = int(max(s.max(), d.max())) + 1
    return s, d, n


# ---------------------------------------------------------- random generators
def barabasi_albert(n: int, m: int, seed: int = 0):
    """Preferential attachment: a star on m+1 nodes, then every new node joins
    m distinct existing nodes drawn with probability proportional to degree
    (uniform draws from the list of edge endpoints)."""
    rng = np.random.default_rng(seed)
    src = list(range(1, m + 1))
    dst = [0] * m
    ends = src + dst
    for v in range(m + 1, n):
        chosen: set[int] = set()
        while len(chosen) < m:
            chosen.add(ends[int(rng.integers(len(ends)))])
        for u in sorted(chosen):
            src.append(v)
            dst.append(u)
            ends.append(v)
            ends.append(u)
    return np.asarray(src, np.int32), np.asarray(dst, np.int32), n


def _rmat_round(rng, scale, count, a, b, c):
    u = np.zeros(count, np.int64)
    v = np.zeros(count, np.int64)
    ab, abc = np.float32(a + b), np.float32(a + b + c)
    a32 = np.float32(a)
    for _ in range(scale):
        r = rng.random(count, dtype=np.float32)
        u <<= 1
        v <<= 1
        u |= r >= ab                              # quadrants c, d: lower half
        v |= ((r >= a32) & (r < ab)) | (r >= abc)  # quadrants b, d: right half
    return u, v


def rmat(scale: int, n_edges: int, a=0.57, b=0.19, c=0.19, seed: int = 1,
         chunk: int = 1 << 24):
    """R-MAT graph on 2^scale nodes with exactly ``n_edges`` unique undirected
    non-loop edges: candidate pairs are drawn in rounds, and the first
    ``n_edges`` distinct pairs in sampling order are kept."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    keys = []
    total = 0
    while True:
        want = int(n_edges * 1.3) + 1024 if total == 0 else max(n_edges // 4, 1024)
        while want > 0:
            cnt = min(want, chunk)
            u, v = _rmat_round(rng, scale, cnt, a, b, c)
            keep = u != v
            u, v = u[keep], v[keep]
            keys.append(np.minimum(u, v) * n + np.maximum(u, v))
            want -= cnt
            total += cnt
        allk = np.concatenate(keys)
        _, first = np.unique(allk, return_index=True)
        if first.size >= n_edges:
            break
        keys = [allk]
    first.sort()
    key = allk[first[:n_edges]]
    lo, hi = key // n, key % n
    # orientation of each stored pair is random (undirected graph)
    flip = rng.random(key.size, dtype=np.float32) < 0.5
    s = np.where(flip, hi, lo).astype(np.int32)
    d = np.where(flip, lo, hi).astype(np.int32)
    return s, d, n


def rmat_torch(scale: int, n_edges: int, a=0.57, b=0.19, c=0.19, seed: int = 1,
               device="cuda", chunk: int = 1 << 26, n_nodes: int | None = None):
    """``rmat`` drawn with torch on ``device``: candidate pairs in rounds, the
    first ``n_edges`` distinct undirected non-loop pairs in sampling order,
    random orientation.  Returns int32 tensors (src, dst) on ``device`` and n.
    ``n_nodes`` (< 2^scale) restricts the graph to nodes [0, n_nodes): pairs
    with an endpoint outside are rejected, the usual way to draw R-MAT graphs
    whose node count is not a power of two."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    n = 1 << scale
    nn = n if n_nodes is None else int(n_nodes)
    if not 1 < nn <= n:
        raise ValueError("n_nodes must lie in (1, 2^scale]")
    ab, abc = a + b, a + b + c
    keys = torch.empty(0, dtype=torch.int64, device=device)
    want = int(n_edges * 1.3 * n / nn) + 1024
    while True:
        parts = [keys]
        while want > 0:
            cnt = min(want, chunk)
            u = torch.zeros(cnt, dtype=torch.int64, device=device)
            v = torch.zeros(cnt, dtype=torch.int64, device=device)
            for _ in range(scale):
                r = torch.rand(cnt, generator=gen, device=device)
                u = (u << 1) | (r >= ab).long()
                v = (v << 1) | (((r >= a) & (r < ab)) | (r >= abc)).long()
            keep = (u != v) & (u < nn) & (v < nn)
            u, v = u[keep], v[keep]
            parts.append(torch.minimum(u, v) * n + torch.maximum(u, v))
            want -= cnt
        keys = torch.cat(parts)
        srt, perm = torch.sort(keys, stable=True)
        first = torch.ones_like(srt, dtype=torch.bool)
        first[1:] = srt[1:] != srt[:-1]
        idx = torch.sort(perm[first]).values
        if idx.numel() >= n_edges:
            break
        want = max(n_edges // 4, 1024)
    key = keys[idx[:n_edges]]
    del keys, srt, perm, first, idx
    lo, hi = key // n, key % n
    flip = torch.rand(key.numel(), generator=gen, device=device) < 0.5
    src = torch.where(flip, hi, lo).to(torch.int32)
    dst = torch.where(flip, lo, hi).to(torch.int32)
    return src, dst, nn


def rewire_torch(src, dst, n: int, frac: float = 1e-3, seed: int = 0):
    """``rewire`` on the device (torch tensors in, int32 tensors out): the
    ceil(frac*|E|) edges to delete are a uniform sample without replacement
    of the sorted unique edges, and the new edges are the first distinct
    uniformly drawn non-loop non-edges in sampling order.  Node set and ids
    are kept."""
    import torch

    dev = src.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    s, d = src.long(), dst.long()
    keys = torch.unique(torch.minimum(s, d) * n + torch.maximum(s, d))  # sorted
    m = keys.numel()
    k = int(math.ceil(frac * m))
    drop = torch.randperm(m, generator=gen, device=dev)[:k]
    keep = torch.ones(m, dtype=torch.bool, device=dev)
    keep[drop] = False
    new = torch.empty(0, dtype=torch.int64, device=dev)
    while new.numel() < k:
        cnt = 4 * (k - new.numel()) + 1024
        a = torch.randint(0, n, (cnt,), generator=gen, device=dev)
        b = torch.randint(0, n, (cnt,), generator=gen, device=dev)
        ok = a != b
        cand = (torch.minimum(a, b) * n + torch.maximum(a, b))[ok]
        pos = torch.searchsorted(keys, cand).clamp(max=m - 1)
        cand = cand[keys[pos] != cand]
        cand = torch.cat([new, cand])
        # first occurrence of each key, in sampling order
        srt, perm = torch.sort(cand, stable=True)
        first = torch.ones_like(srt, dtype=torch.bool)
        first[1:] = srt[1:] != srt[:-1]
        new = cand[torch.sort(perm[first]).values]
    allk = torch.cat([keys[keep], new[:k]])
    return (allk // n).to(torch.int32), (allk % n).to(torch.int32), n


def erdos_renyi(n: int, p: float, seed: int = 0):
    rng = np.random.default_rng(seed)
    i, j = np.triu_indices(n, 1)
    keep = rng.random(i.size) < p
    return i[keep].astype(np.int32), j[keep].astype(np.int32), n


def _tri_pair(idx, m):
    """Pair (i, j), i < j < m, of row-major index idx in the strict upper triangle."""
    idx = np.asarray(idx, np.int64)
    b = 2 * m - 1
    i = np.floor((b - np.sqrt(b * b - 8.0 * idx)) / 2).astype(np.int64)
    # guard floating-point rounding of the closed form
    start = i * (2 * m - i - 1) // 2
    low = idx < start
    i[low] -= 1
    start = i * (2 * m - i - 1) // 2
    nxt = (i + 1) * (2 * m - i - 2) // 2
    high = idx >= nxt
    i[high] += 1
    start = i * (2 * m - i - 1) // 2
    j = idx - start + i + 1
    return i, j


def sbm(sizes, p_in: float, p_out: float, seed: int = 0):
    """Stochastic block model with the given block sizes: for every pair of
    blocks the number of edges is Binomial(pairs, p) and the edges are that
    many distinct pairs drawn uniformly."""
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes, np.int64)
    start = np.concatenate([[0], np.cumsum(sizes)])
    n = int(start[-1])
    us, vs = [], []
    for a in range(sizes.size):
        for b in range(a, sizes.size):
            sa, sb = int(sizes[a]), int(sizes[b])
            pairs = sa * (sa - 1) // 2 if a == b else sa * sb
            if pairs == 0:
                continue
            k = int(rng.binomial(pairs, p_in if a == b else p_out))
            if k == 0:
                continue
            idx = rng.choice(pairs, size=k, replace=False)
            if a == b:
                i, j = _tri_pair(idx, sa)
            else:
                i, j = idx // sb, idx % sb
            us.append(start[a] + i)
            vs.append(start[b] + j)
    if not us:
        return np.zeros(0, np.int32), np.zeros(0, np.int32), n
    return np.concatenate(us).astype(np.int32), np.concatenate(vs).astype(np.int32), n


def sbm_batch(n_graphs: int, seed: int = 3, median: float = 300.0,
              sigma: float = 1.0, lo: int = 10, hi: int = 5000):
    """Batch of SBM graphs: node counts lognormal(ln median, sigma) clipped to
    [lo, hi]; 2-6 blocks as equal as possible; p_in ~ U[0.05, 0.3];
    p_out = p_in / U[5, 20].  Graph g uses seed ``seed + g``."""
    return [sbm_batch_graph(g, seed, median, sigma, lo, hi) for g in range(n_graphs)]


def sbm_batch_graph(g: int, seed: int = 3, median: float = 300.0, sigma: float = 1.0,
                    lo: int = 10, hi: int = 5000):
    """Graph g of ``sbm_batch(..., seed, ...)`` on its own (it depends on
    seed + g only)."""
    rng = np.random.default_rng(seed + g)
    n = int(np.clip(round(rng.lognormal(np.log(median), sigma)), lo, hi))
    nb = int(rng.integers(2, 7))
    base, rem = divmod(n, nb)
    sizes = [base + (1 if k < rem else 0) for k in range(nb)]
    p_in = float(rng.uniform(0.05, 0.3))
    p_out = p_in / float(rng.uniform(5.0, 20.0))
    return sbm(sizes, p_in, p_out, seed=seed + g + 1_000_000)


def rewire(src, dst, n: int, frac: float = 1e-3, seed: int = 0):
    """Copy of an undirected simple graph with ceil(frac*|E|) edges rewired:
    each chosen edge is deleted and a uniformly random non-loop non-edge is
    inserted.  Node set and ids are kept."""
    rng = np.random.default_rng(seed)
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    lo, hi = np.minimum(s, d), np.maximum(s, d)
    keys = np.unique(lo * n + hi)
    m = keys.size
    k = int(np.ceil(frac * m))
    drop = rng.choice(m, size=k, replace=False)
    keep = np.ones(m, bool)
    keep[drop] = False
    present = set(keys.tolist()) if m < 5_000_000 else None
    kept = keys[keep]
    new = []
    existing = present if present is not None else set(keys.tolist())
    while len(new) < k:
        a, b = rng.integers(0, n, size=2)
        if a == b:
            continue
        key = int(min(a, b)) * n + int(max(a, b))
        if key in existing:
            continue
        existing.add(key)
        new.append(key)
    allk = np.concatenate([kept, np.asarray(new, np.int64)])
    return (allk // n).astype(np.int32), (allk % n).astype(np.int32), n
