"""Autotuner for the decode: picks the cooperation width G, the encode-time
block size and the lanes per SM (resident CTAs per SM of the persistent
launch, and the size of its work ranges).

The paper's effective-workload law (Sec. III-A, Table I) ties throughput
to lanes = G x N_blocks: starved below ~32K lanes, about half of saturated
near 65K, saturated above ~1M.  The tuner ranks the candidate
(G, block size) pairs by that law, measures the most promising ones on the
GPU (CUDA events, median of several decodes), and returns the fastest.
"""
from __future__ import annotations

import math

import numpy as np

from . import aclz

# normalised throughput against lanes, read off Table I (log-linear between)
_TABLE_I = ((32_768, 0.31), (65_536, 0.525), (131_072, 0.81), (1_048_576, 1.0))


def lanes_law(lanes: float) -> float:
    """Predicted normalised throughput for a lane count (Table I)."""
    if lanes <= _TABLE_I[0][0]:
        return _TABLE_I[0][1] * lanes / _TABLE_I[0][0]
    for (l0, v0), (l1, v1) in zip(_TABLE_I, _TABLE_I[1:]):
        if lanes <= l1:
            f = (math.log(lanes) - math.log(l0)) / (math.log(l1) - math.log(l0))
            return v0 + f * (v1 - v0)
    return 1.0


def measure(h: int, out, reps: int = 5, warmup: int = 2, stream=None, **cfg) -> float:
    """Median milliseconds of one decode_all with this configuration."""
    import torch
    st = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        aclz.aclz_decode_all(h, out, stream=st, **cfg)
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        aclz.aclz_decode_all(h, out, stream=st, **cfg)
        b.record(st)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    if aclz.aclz_device_status(h, st) != aclz.ACLZ_OK:
        raise RuntimeError("decode reported a device error during tuning")
    return float(np.median(ms))


def tune(build, total: int, block_sizes=(8192, 16384, 32768, 65536, 131072), Gs=(8, 16, 32),
         ctas=(0, 2), range_bytes=(8192, 20480), top: int = 4, reps: int = 5, stream=None) -> dict:
    """build(block_size) -> container bytes of the same data at that block
    size; total = the data's bytes (GB/s are total / time).  Returns
    {"best": {...}, "trials": [...]}."""
    import torch
    cands = []
    for bs in block_sizes:
        nb = -(-total // bs)
        for G in Gs:
            cands.append((lanes_law(G * nb), bs, G))
    cands.sort(key=lambda c: (-c[0], -c[2]))
    keep = {}
    for pred, bs, G in cands:
        keep.setdefault(bs, []).append((pred, G))
    # the `top` best-predicted block sizes, each with its best-predicted G
    chosen = sorted(((max(v)[0], bs, max(v)[1]) for bs, v in keep.items()), reverse=True)[:top]
    trials = []
    out = None
    st = stream or torch.cuda.current_stream()
    for pred, bs, G in chosen:
        c = build(bs)
        h = aclz.aclz_upload(c, st)
        try:
            info = aclz.aclz_handle_info(h)
            # a merged batch is longer than its streams (block-aligned bases)
            need = max(16, (int(info.total_len) + 15) // 16 * 16)
            if out is None or out.numel() < need:
                out = torch.empty(need, dtype=torch.uint8, device="cuda")
            for G2 in sorted({G, 32}):
                for cps in ctas:
                    for rb in range_bytes:
                        aclz.aclz_set_range_bytes(h, rb, st)
                        ms = measure(h, out, reps=reps, stream=st, G=G2, ctas_per_sm=cps)
                        trials.append(dict(block_size=bs, G=G2, ctas_per_sm=cps, range_bytes=rb,
                                           lanes=G2 * info.n_blocks, predicted=round(lanes_law(G2 * info.n_blocks), 3),
                                           ms=round(ms, 4), gbs=round(total / ms / 1e6, 1)))
        finally:
            aclz.aclz_free(h)
    best = max(trials, key=lambda t: t["gbs"])
    return {"best": best, "trials": trials}
