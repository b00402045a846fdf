"""Timing of the GPU tile entropy stage against the match phase it feeds.

The paper puts a tile-ANS stage (64 KB tiles decoded many at a time) in
front of the match kernel and reports the full pipeline's time as about 9%
entropy decode and 91% match phase (Sec. II; Sec. V).  Here a v1 container
is coded into the ACLE form (order-0 rANS over 64 KiB tiles of its 16
token byte planes and its literals), uploaded with aclz_upload_acle_ev, and
the device tile decode (k_ans_tiles, then k_planes_to_tokens) is timed by
CUDA events around it; the match-phase decode of the same handle is timed
the same way.  Throughput of the tile stage is given as ACLE payload bytes
read plus decoded plane and literal bytes written, per second, beside the
measured HBM peak.

    python -m paper_2607_18541_gb300.tiles [--mib 1024] [--stream fastq|copy] [--reps 5]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics

import numpy as np

from . import aclz, learned, synth


def build(stream: str, mib: int):
    """(v1 container, decoded length) of the named workload."""
    n = mib << 20
    if stream == "fastq":
        x = synth.fastq(n, seed=synth.SEED_FASTQ)
        return learned.encode(x, (12, 16, 24, 32), block_size=1 << 14), n
    sw = synth.copy_sweep(n, 1 << 15, 1024, seed=synth.SEED_COPY + 1024)
    c = aclz.aclz_pack(sw.total, sw.block_size, (4, 4, 4, 4), sw.blk_ntok, sw.lit_len, sw.match_len, sw.src,
                       sw.literals)
    return c, n


def hbm_peak() -> float:
    p = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"])
    return 6800.0


def run(stream: str, mib: int, reps: int) -> dict:
    import torch
    c, n = build(stream, mib)
    e = aclz.aclz_acle_encode(c)
    info = aclz.aclz_container_info(c)
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    ev1.record(st)
    st.synchronize()
    tile_ms, match_ms = [], []
    out = torch.empty((n + 15) // 16 * 16, dtype=torch.uint8, device="cuda")
    expect = None
    for i in range(reps + 1):
        h = ctypes.c_void_p(0)
        rc = aclz.lib().aclz_upload_acle_ev(e.ctypes.data, e.size, 0, ctypes.c_void_p(st.cuda_stream),
                                            ctypes.byref(h), ctypes.c_void_p(ev0.cuda_event),
                                            ctypes.c_void_p(ev1.cuda_event))
        if rc:
            raise aclz.AclzError(rc, "aclz_upload_acle_ev")
        hh = int(h.value)
        try:
            st.synchronize()
            t_tiles = ev0.elapsed_time(ev1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            aclz.aclz_decode_all(hh, out, stream=st)
            b.record(st)
            st.synchronize()
            if aclz.aclz_device_status(hh, st) != aclz.ACLZ_OK:
                raise RuntimeError("decode reported a device error")
            f = aclz.aclz_fnv(out, n, stream=st)
            if expect is None:
                expect = f
            elif f != expect:
                raise RuntimeError("decodes of the same container differ")
            if i:
                tile_ms.append(t_tiles)
                match_ms.append(a.elapsed_time(b))
        finally:
            aclz.aclz_free(hh)
    # the ACLE decode must give the v1 container's decode
    h = aclz.aclz_upload(c, st)
    try:
        aclz.aclz_decode_all(h, out, stream=st)
        if aclz.aclz_fnv(out, n, stream=st) != expect:
            raise RuntimeError("ACLE upload decodes differently from the v1 container")
    finally:
        aclz.aclz_free(h)
    t = statistics.median(tile_ms)
    m = statistics.median(match_ms)
    moved = int(e.size) + 16 * info.n_tokens + info.n_literals
    peak = hbm_peak()
    return {"stream": stream, "mib": mib, "v1_bytes": int(c.size), "acle_bytes": int(e.size),
            "ratio_acle": round(n / e.size, 4), "tokens": int(info.n_tokens), "literals": int(info.n_literals),
            "tiles_ms": round(t, 4), "tiles_gbs_moved": round(moved / (t * 1e-3) / 1e9, 1),
            "tiles_frac_of_hbm": round(moved / (t * 1e-3) / 1e9 / peak, 4),
            "tiles_output_gbs": round(n / (t * 1e-3) / 1e9, 1),
            "match_ms": round(m, 4), "match_output_gbs": round(n / (m * 1e-3) / 1e9, 1),
            "entropy_share": round(t / (t + m), 4), "reps": reps,
            "paper_split": "ANS 9% / match 91% (Sec. V)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mib", type=int, default=1024)
    ap.add_argument("--stream", default="fastq,copy")
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    for s in args.stream.split(","):
        print(json.dumps(run(s, args.mib, args.reps)), flush=True)


if __name__ == "__main__":
    main()
