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

    def __init__(self, containers, stream=None, device=None, flatten: bool = False):
        import torch
        self.merged, self.offsets = aclz.aclz_batch_merge(containers)
        self.lengths = np.array([aclz.aclz_container_info(c).total_len for c in containers], dtype=np.uint64)
        self.stream = stream
        self.h = aclz.aclz_upload(self.merged, stream, flags=aclz.ACLZ_UPLOAD_FLATTEN if flatten else 0)
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


def main():
    """Full-size batched benchmark: 4096 streams, output sizes log-uniform
    16 KiB - 64 MiB (half Markov bytes, half FASTQ-like), encoded at
    12/16/24/32; block size, G, CTAs per SM and range size tuned on a sample
    of the streams; then one graph-captured batched decode of all streams
    against the same containers decoded one at a time.  Prints JSON lines."""
    import argparse
    import json
    import torch
    from . import autotune
    ap = argparse.ArgumentParser()
    ap.add_argument("--streams", type=int, default=4096)
    ap.add_argument("--lo", type=int, default=16 << 10)
    ap.add_argument("--hi", type=int, default=64 << 20)
    ap.add_argument("--chain-depth", type=int, default=1)
    ap.add_argument("--tune-sample", type=int, default=256)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    t0 = time.time()
    streams = make_streams(a.streams, a.lo, a.hi)
    total = int(sum(x.size for x in streams))
    t_gen = time.time() - t0

    def params(bs):
        p = aclz.aclz_encode_params_default(aclz.ACLZ_PRESET_TUNED)
        p.block_size = bs
        p.chain_depth = a.chain_depth
        return p

    step = max(1, a.streams // a.tune_sample)
    sample = streams[::step]
    t0 = time.time()
    tuned = autotune.tune(lambda bs: aclz.aclz_batch_merge(encode_streams(sample, params(bs)))[0],
                          int(sum(x.size for x in sample)), block_sizes=(16384, 32768, 65536, 131072),
                          top=3, reps=3)
    best = tuned["best"]
    t_tune = time.time() - t0
    print(json.dumps({"tuned_on_streams": len(sample), "best": best, "tune_s": round(t_tune, 1)}), flush=True)
    t0 = time.time()
    cs = encode_streams(streams, params(best["block_size"]))
    t_enc = time.time() - t0
    cfg = dict(G=best["G"], ctas_per_sm=best["ctas_per_sm"])
    st = torch.cuda.current_stream()
    dec = BatchDecoder(cs, stream=st)
    try:
        aclz.aclz_set_range_bytes(dec.h, best["range_bytes"], st)
        info = aclz.aclz_handle_info(dec.h)
        ms_b = time_batched(dec, reps=a.reps, graph=True, **cfg)
        if aclz.aclz_device_status(dec.h, st) != aclz.ACLZ_OK:
            raise RuntimeError("batched decode reported a device error")
        exact = 0
        for i, x in enumerate(streams):
            exact += bool(torch.equal(dec.stream_output(i), torch.from_numpy(x).to("cuda", non_blocking=True)))
        row_b = dict(form="batched: one persistent graph-captured launch", streams=len(streams), bytes=total,
                     blocks=info.n_blocks, waves=info.n_waves, lanes=best["G"] * info.n_blocks,
                     ms=round(ms_b, 3), gbs=round(total / ms_b / 1e6, 1), exact_streams=exact, **cfg,
                     block_size=best["block_size"], range_bytes=best["range_bytes"])
    finally:
        dec.close()
    print(json.dumps(row_b), flush=True)
    # the same batch with the flattened two-wave schedule
    t0 = time.time()
    dec = BatchDecoder(cs, stream=st, flatten=True)
    t_up = time.time() - t0
    try:
        ms_f = time_batched(dec, reps=a.reps, graph=True, **cfg)
        if aclz.aclz_device_status(dec.h, st) != aclz.ACLZ_OK:
            raise RuntimeError("flattened batched decode reported a device error")
        exact_f = sum(bool(torch.equal(dec.stream_output(i), torch.from_numpy(x).to("cuda", non_blocking=True)))
                      for i, x in enumerate(streams))
        info_f = aclz.aclz_handle_info(dec.h)
        print(json.dumps(dict(form="batched, flattened schedule (two waves)", streams=len(streams), bytes=total,
                              pieces=info_f.n_deferred, ms=round(ms_f, 3), gbs=round(total / ms_f / 1e6, 1),
                              exact_streams=exact_f, upload_s=round(t_up, 2), **cfg)), flush=True)
    finally:
        dec.close()
    ms_1, outs = time_one_by_one(cs, stream=st, reps=1, **cfg)
    exact1 = sum(bool(torch.equal(o[:x.size], torch.from_numpy(x).to("cuda"))) for o, x in zip(outs, streams))
    del outs
    print(json.dumps(dict(form="one stream at a time (single-stream decode)", streams=len(streams), bytes=total,
                          ms=round(ms_1, 3), gbs=round(total / ms_1 / 1e6, 2), exact_streams=exact1,
                          gen_s=round(t_gen, 1), encode_s=round(t_enc, 1), chain_depth=a.chain_depth)),
          flush=True)


if __name__ == "__main__":
    main()
