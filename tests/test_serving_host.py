"""Host side of the serving forms (no GPU): the batched workload's streams
follow their recipe (log-uniform sizes in range, Markov bytes at even
indices, FASTQ-like text at odd ones, reproducible), the per-thread encode
of a batch equals encoding each stream alone and decodes (oracle) to it,
the merged container of a batch holds every stream at its offset, and the
serving loop's latency summary is the plain percentile of the samples."""
import numpy as np

import oracle
from paper_2607_18541_gb300 import aclz, batched, serve, synth
from paper_2607_18541_gb300 import build as libbuild


def test_batch_streams_follow_the_recipe():
    s1 = batched.make_streams(24, 1 << 10, 1 << 16, seed=81, threads=3)
    s2 = batched.make_streams(24, 1 << 10, 1 << 16, seed=81, threads=1)
    assert all(np.array_equal(a, b) for a, b in zip(s1, s2))
    sizes = np.array([s.size for s in s1])
    assert sizes.min() >= 1 << 10 and sizes.max() <= 1 << 16
    for i, s in enumerate(s1):
        if i % 2:  # FASTQ-like: records start with '@'
            assert s[0] == ord("@")
        else:      # Markov bytes over 0x30-0x6F
            assert s.min() >= 0x30 and s.max() <= 0x6F


def test_batch_encode_and_merge_hold_every_stream():
    libbuild.build()
    streams = batched.make_streams(9, 1 << 12, 1 << 15, seed=82, threads=2)
    p = aclz.aclz_encode_params_default(aclz.ACLZ_PRESET_TUNED)
    p.block_size = 1 << 12
    cs = batched.encode_streams(streams, p, threads=3)
    for s, c in zip(streams, cs):
        assert np.array_equal(c, aclz.aclz_encode(s, p))
        assert np.array_equal(oracle.decode(c), s)
    merged, offs = aclz.aclz_batch_merge(cs)
    out = oracle.decode(merged)
    for s, o in zip(streams, offs):
        assert np.array_equal(out[int(o):int(o) + s.size], s)


def test_latency_summary_is_the_percentile():
    lat = np.random.default_rng(83).exponential(0.002, 1000)
    r = serve.percentiles(lat)
    assert abs(r["p50_ms"] - np.percentile(lat, 50) * 1e3) < 1e-3
    assert abs(r["p99_ms"] - np.percentile(lat, 99) * 1e3) < 1e-3
    assert abs(r["mean_ms"] - lat.mean() * 1e3) < 1e-3
