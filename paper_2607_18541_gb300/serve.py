"""Continuous-batching request loop for range decodes (seek) against a
device-resident compressed corpus.

Requests arrive over time (Poisson); each asks for decode(corpus)[lo, hi).
Every tick the loop retires finished batches (returning their output memory
to the budget), admits queued requests in arrival order while their output
buffers fit in the free-HBM budget and the in-flight slots, and launches the
newly admitted ones together in one range-decode launch on the next of
several CUDA streams, so batches that arrive while others run overlap on the
device.  Latency = completion - arrival takes each term from its own clock:
arrivals are host times from the start of the run, completions are CUDA
event times from an event recorded, and waited for, just before the run
starts.  The event therefore precedes the host start by at most the time
that wait took (reported as clock_bias_ms), so a latency is overstated by at
most that much and is never understated.

In the paper a seek reads any region of a stream that stays compressed in
GPU memory, decoding only that region (abstract; Sec. I); this loop serves
many such region reads at once.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from collections import deque

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2607_18541_gb300 import aclz, synth  # noqa: E402
else:
    from . import aclz, synth

REQ_BYTES = 32


def build_corpus(total: int, seed: int = synth.SEED_SERVE, block_size: int = 1 << 16,
                 preset: int = aclz.ACLZ_PRESET_TUNED, window: int = 1 << 30, chain_depth: int = 8):
    """Order-3 Markov word text of `total` bytes and its container (64 KiB
    blocks, 12/16/24/32, matches within 1 GiB; a shallow hash chain keeps
    host encoding of multi-GiB text to minutes)."""
    x = synth.wordtext(total, seed=seed)
    p = aclz.aclz_encode_params_default(preset)
    p.block_size = block_size
    p.window = window
    p.chain_depth = chain_depth
    return x, aclz.aclz_encode(x, p)


class Server:
    def __init__(self, handle: int, budget_bytes: int, max_inflight: int = 256, n_streams: int = 4,
                 max_batch: int = 512):
        import torch
        self.torch = torch
        self.h = handle
        self.budget = int(budget_bytes)
        self.max_inflight = max_inflight
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.next_stream = 0

    def run(self, arrivals, starts, sizes, keep_outputs: bool = False, on_done=None):
        """Serve requests i = 0..n-1 arriving at arrivals[i] seconds (from
        the start of the run).  Returns per-request latency (s), makespan,
        and optionally the outputs (host copies).  on_done(i, buf), when
        given, sees each result's device buffer as its batch retires."""
        torch = self.torch
        n = len(arrivals)
        order = np.argsort(arrivals, kind="stable")
        queue = deque()
        inflight = []  # (event, idx list, buffers, req table, bytes)
        used = 0
        done_t = np.full(n, np.nan)
        outputs = {} if keep_outputs else None
        t_start_ev = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t_start_ev.record(torch.cuda.current_stream())
        tw = time.perf_counter()
        t_start_ev.synchronize()  # the event precedes t0 by at most this wait
        t0 = time.perf_counter()
        self.clock_bias_s = t0 - tw
        nxt = 0
        served = 0
        while served < n:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[order[nxt]] <= now:
                queue.append(int(order[nxt]))
                nxt += 1
            # retire finished batches
            still = []
            for ev, idx, bufs, table, nbytes in inflight:
                if ev.query():
                    tdone = t_start_ev.elapsed_time(ev) * 1e-3
                    for i, b in zip(idx, bufs):
                        done_t[i] = tdone
                        if keep_outputs:
                            outputs[i] = b[:int(sizes[i])].cpu().numpy()
                        if on_done is not None:
                            on_done(i, b)
                    used -= nbytes
                    served += len(idx)
                else:
                    still.append((ev, idx, bufs, table, nbytes))
            inflight = still
            # admit in arrival order while memory and slots allow
            batch = []
            n_inflight = sum(len(x[1]) for x in inflight)
            while queue and len(batch) < self.max_batch and n_inflight + len(batch) < self.max_inflight:
                i = queue[0]
                need = (int(sizes[i]) + 15) // 16 * 16 + REQ_BYTES
                if used + need > self.budget and (inflight or batch):
                    break
                queue.popleft()
                batch.append(i)
                used += need
            if batch:
                st = self.streams[self.next_stream]
                self.next_stream = (self.next_stream + 1) % len(self.streams)
                table = torch.empty(len(batch) * REQ_BYTES, dtype=torch.uint8).pin_memory()
                tv = table.numpy().view(np.uint64).reshape(len(batch), 4)
                bufs = []
                with torch.cuda.stream(st):
                    for k, i in enumerate(batch):
                        b = torch.empty(max(16, (int(sizes[i]) + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
                        bufs.append(b)
                        tv[k, 0] = starts[i]
                        tv[k, 1] = starts[i] + sizes[i]
                        tv[k, 2] = b.data_ptr()
                        tv[k, 3] = 0
                    aclz.aclz_decode_ranges_async(self.h, len(batch), table.data_ptr(), st)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(st)
                nbytes = sum((int(sizes[i]) + 15) // 16 * 16 + REQ_BYTES for i in batch)
                inflight.append((ev, batch, bufs, table, nbytes))
            elif not inflight and nxt < n:
                # idle: sleep until the next arrival
                time.sleep(max(0.0, min(1e-3, arrivals[order[nxt]] - (time.perf_counter() - t0))))
            else:
                time.sleep(20e-6)
        torch.cuda.synchronize()
        lat = done_t - np.asarray(arrivals)
        makespan = float(np.nanmax(done_t)) - float(np.min(arrivals)) if n else 0.0
        return lat, makespan, outputs


def percentiles(lat_s) -> dict:
    lat = np.asarray(lat_s) * 1e3
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3)}


def serve_benchmark(h: int, corpus_len: int, n_requests: int, loads=(0.25, 0.5, 0.75, 0.9),
                    lo: int = 16 << 10, hi: int = 256 << 20, seed: int = synth.SEED_SERVE + 7,
                    budget_frac: float = 0.8):
    """Saturated throughput first (all requests at t = 0), then Poisson
    arrivals at the given fractions of it.  Returns a list of result rows."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * budget_frac)
    srv = Server(h, budget)
    mean_size = (hi - lo) / np.log(hi / lo)
    rows = []
    _, st, sz = synth.requests(n_requests, 1.0, lo, min(hi, corpus_len), corpus_len, seed)
    zero = np.zeros(n_requests)
    lat, span, _ = srv.run(zero, st, sz)
    sat_bps = float(sz.sum()) / span
    rows.append(dict(load="saturated", requests=n_requests, gbs=round(sat_bps / 1e9, 2),
                     clock_bias_ms=round(srv.clock_bias_s * 1e3, 4), **percentiles(lat)))
    for f in loads:
        rate = f * sat_bps / mean_size
        arr, st, sz = synth.requests(n_requests, rate, lo, min(hi, corpus_len), corpus_len, seed + int(f * 100))
        lat, span, _ = srv.run(arr, st, sz)
        rows.append(dict(load=f, offered_req_per_s=round(rate, 2), requests=n_requests,
                         gbs=round(float(sz.sum()) / span / 1e9, 2), clock_bias_ms=round(srv.clock_bias_s * 1e3, 4),
                         **percentiles(lat)))
    return rows


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--corpus-gib", type=float, default=8.0)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--loads", default="0.25,0.5,0.75,0.9")
    ap.add_argument("--max-size", type=int, default=256 << 20)
    ap.add_argument("--chain-depth", type=int, default=4)
    a = ap.parse_args()
    total = int(a.corpus_gib * (1 << 30))
    t0 = time.time()
    x, c = build_corpus(total, chain_depth=a.chain_depth)
    t_build = time.time() - t0
    # range decode does not use wave tags: the flattening upload skips the
    # ordered minimal-tag pass, which is slow on word text's deep chains
    t0 = time.time()
    h = aclz.aclz_upload(c, torch.cuda.current_stream(), flags=aclz.ACLZ_UPLOAD_FLATTEN)
    t_up = time.time() - t0
    try:
        info = aclz.aclz_handle_info(h)
        rows = serve_benchmark(h, total, a.requests, tuple(float(v) for v in a.loads.split(",")),
                               hi=a.max_size)
        for r in rows:
            r.update(corpus_bytes=total, container_bytes=int(c.size), block_size=info.block_size,
                     chain_depth=a.chain_depth, build_s=round(t_build, 1), upload_s=round(t_up, 2))
            print(json.dumps(r), flush=True)
    finally:
        aclz.aclz_free(h)


if __name__ == "__main__":
    main()
