"""Pins of the probe generator: the published SplitMix64 stream and the
properties Eq. trace needs (zero mean, unit variance, +-1 entries)."""
import numpy as np

import synth
from oracle import probes
from oracle.laplacian import build_laplacian

# First outputs of SplitMix64 seeded with 0 (Vigna's reference splitmix64.c;
# Steele, Lea, Flood, OOPSLA 2014).
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_splitmix64_stream():
    out = probes.raw(0, 0, 0, np.arange(4))
    assert [int(x) for x in out] == SPLITMIX64_SEED0
    # signs are bit 63: 0xE2.. -> -1, 0x6E.. -> +1, 0x06.. -> +1, 0xF8.. -> -1
    assert probes.rademacher(0, 0, 0, np.arange(4)).tolist() == [-1.0, 1.0, 1.0, -1.0]


def test_fields_are_distinct_streams():
    node = np.arange(4096)
    a = probes.rademacher(5, 0, 0, node)
    b = probes.rademacher(5, 0, 1, node)
    c = probes.rademacher(5, 1, 0, node)
    d = probes.rademacher(6, 0, 0, node)
    for x in (b, c, d):
        assert 0.3 < np.mean(a != x) < 0.7


def test_zero_mean_unit_variance():
    n = 1 << 16
    for p in range(8):
        v = probes.rademacher(123, 0, p, np.arange(n))
        assert set(np.unique(v)) == {-1.0, 1.0}
        assert abs(v.mean()) < 4 / np.sqrt(n)
        assert v @ v == n


def test_signs_follow_original_ids():
    s, d, n = synth.disjoint_union(synth.cycle(5), synth.path(4), extra_isolated=0)
    s = np.where(s >= 5, s + 3, s).astype(np.int32)   # ids 5,6,7 become isolated
    d = np.where(d >= 5, d + 3, d).astype(np.int32)
    lap = build_laplacian(s, d, 12, drop_isolated=True)
    full = probes.probe_block(9, 0, 3, np.arange(12))
    kept = probes.probe_block(9, 0, 3, lap.old_id)
    assert np.array_equal(full[lap.old_id], kept)
