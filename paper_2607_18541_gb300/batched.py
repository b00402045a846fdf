"""Batched decode of many independent compressed streams in one launch.

Streams are merged into one container whose stream i starts on a block
boundary (``aclz_batch_merge``: sources rebased, streams never reference one
another), so the persistent decode schedules the (stream, block, wave) work of
every stream in one wave-major list and one cooperative launch, captured in a
CUDA graph.  The lanes law of Sec. III-A is why this pays: a small stream alone
has too few G-lane groups to fill the GPU, thousands of them together do.

The comparison point is the same streams decoded one at a time with the
single-stream decode.
"""
from __future__ import annotations

import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import aclz, synth


def make_streams(n: int, lo: int, hi: int, seed: int = synth.SEED_BATCH, threads: int = 0):
    """n streams with output sizes log-uniform in [lo, hi]; even index order-2
    Markov bytes (one shared model, per-stream sequence seed), odd index
    FASTQ-like text."""
    sizes, seeds = synth.stream_sizes(n, lo, hi, seed)
    model = synth.MarkovModel(seed)
    threads = threads or min(16, os.cpu_count() or 1)

    def gen(i):
        return synth.batch_stream(i, int(sizes[i]), int(seeds[i]), model)

    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(gen, range(n)))


def encode_streams(streams, params, block_min_match=None, threads: int = 0):
    """Encode every stream with the library's host encoder (one stream per
    worker thread)."""
    threads = threads or min(16, os.cpu_count() or 1)

    def enc(i):
        bmm = None if block_min_match is None else block_min_match[i]
        return aclz.aclz_encode(streams[i], params, block_min_match=bmm, threads=1)

    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(enc, range(len(streams))))


class BatchDecoder:
    """One merged, uploaded batch and its output buffer."""

    def __init__(self, containers, stream=None, device=None):
        import torch
        self.merged, self.offsets = aclz.aclz_batch_merge(containers)
        self.lengths = np.array([aclz.aclz_container_info(c).total_len for c in containers], dtype=np.uint64)
        self.stream = stream
        self.h = aclz.aclz_upload(self.merged, stream)
        info = aclz.aclz_handle_info(self.h)
        self.total = int(info.total_len)
        self.out = torch.empty(max(16, (self.total + 15) // 16 * 16), dtype=torch.uint8,
                               device=device or "cuda")
        self.graph = None

    def decode(self, **cfg) -> None:
        aclz.aclz_decode_all(self.h, self.out, stream=self.stream, **cfg)

    def capture(self, **cfg) -> None:
        if self.graph:
            aclz.aclz_graph_free(self.graph)
        self.graph = aclz.aclz_graph_create(self.h, self.out, stream=self.stream, **cfg)

    def replay(self) -> None:
        aclz.aclz_graph_launch(self.graph, self.stream)

    def stream_output(self, i: int):
        o, n = int(self.offsets[i]), int(self.lengths[i])
        return self.out[o:o + n]

    def close(self) -> None:
        if self.graph:
            aclz.aclz_graph_free(self.graph)
            self.graph = None
        if self.h:
            aclz.aclz_free(self.h)
            self.h = 0


def time_batched(dec: BatchDecoder, reps: int = 10, warmup: int = 3, graph: bool = True, **cfg) -> float:
    """Median ms of one batched decode (graph replay when graph)."""
    import torch
    st = dec.stream or torch.cuda.current_stream()
    if graph:
        dec.capture(**cfg)
    run = dec.replay if graph else (lambda: dec.decode(**cfg))
    for _ in range(warmup):
        run()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        run()
        b.record(st)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.median(ms))


def time_one_by_one(containers, stream=None, reps: int = 3, **cfg):
    """Single-stream decode of every stream in turn (each uploaded once,
    outside the timing); returns (median ms of the whole sequence, outputs)."""
    import torch
    st = stream or torch.cuda.current_stream()
    hs, outs = [], []
    try:
        for c in containers:
            h = aclz.aclz_upload(c, st)
            n = int(aclz.aclz_handle_info(h).total_len)
            hs.append(h)
            outs.append(torch.empty(max(16, (n + 15) // 16 * 16), dtype=torch.uint8, device="cuda"))
        for h, o in zip(hs, outs):
            aclz.aclz_decode_all(h, o, stream=st, **cfg)
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for h, o in zip(hs, outs):
                aclz.aclz_decode_all(h, o, stream=st, **cfg)
            b.record(st)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms)), outs
    finally:
        for h in hs:
            aclz.aclz_free(h)
