"""Rademacher probe vectors (test infrastructure; see package header).

Eq. trace (Sec. 3.1) needs n_v random vectors with zero mean and unit
variance; the text allows Rademacher vectors.  The paper does not fix a
generator.  Reading: each sign comes from the SplitMix64 output function
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) applied to the counter state

    x = seed + gamma * (c + 1),    c = graph << 48 | probe << 32 | node,

with gamma = 0x9E3779B97F4A7C15, so that graph 0, probe 0, nodes 0, 1, 2, ...
walk the ordinary SplitMix64 stream of ``seed``.  The sign is -1 where bit 63
of the output is set, +1 otherwise.  ``node`` is the ORIGINAL node id, so
dropping isolated nodes leaves every kept node's sign unchanged.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 states (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def counter(graph: int, probe: int, node) -> np.ndarray:
    node = np.asarray(node, dtype=np.uint64)
    return (np.uint64(graph) << np.uint64(48)) | (np.uint64(probe) << np.uint64(32)) | node


def raw(seed: int, graph: int, probe: int, node) -> np.ndarray:
    c = counter(graph, probe, node)
    with np.errstate(over="ignore"):
        x = np.uint64(seed) + GAMMA * (c + np.uint64(1))
    return splitmix64_mix(x)


def rademacher(seed: int, graph: int, probe: int, node_ids) -> np.ndarray:
    """+-1.0 (float64) for each original node id."""
    bits = raw(seed, graph, probe, node_ids) >> np.uint64(63)
    return 1.0 - 2.0 * bits.astype(np.float64)


def probe_block(seed: int, graph: int, n_v: int, node_ids) -> np.ndarray:
    """V[i, p] = sign for kept node i (original id node_ids[i]) and probe p."""
    return np.stack([rademacher(seed, graph, p, node_ids) for p in range(n_v)], axis=1)
