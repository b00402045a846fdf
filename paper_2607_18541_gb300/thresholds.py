"""Threshold variants as fixed configurations (the margin finding of
Sec. IV-C and the limits section): the base 6/8/10/12, the tuned
12/16/24/32 and the pushed 16/24/32/48 minimum match lengths by distance
class (d < 128, < 16384, < 2097152, beyond; Sec. IV-B), and a band sweep
that raises one distance class at a time from the tuned to the pushed
value, to see which band moves the ratio.

For each stream and vector: the entropy-coded size (the ACLE form written
by the library's tile coder, so the ratio is a real coded size, not an
estimate), the order-0 estimate of the same container, tokens, matches and
their mean length, and, on a GPU, the decode throughput of the plain and
the flattened schedules.

    python -m paper_2607_18541_gb300.thresholds [--mib 64] [--gpu] [--streams fastq] [--presets-only]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import aclz, learned, synth

BASE = (6, 8, 10, 12)
TUNED = (12, 16, 24, 32)
PUSHED = (16, 24, 32, 48)


def variants():
    """(name, vector): the three presets, then the tuned vector with one
    distance class raised to its pushed value."""
    out = [("base", BASE), ("tuned", TUNED), ("pushed", PUSHED)]
    for k in range(4):
        v = list(TUNED)
        v[k] = PUSHED[k]
        out.append((f"tuned+band{k}", tuple(v)))
    return out


def streams(mib: int):
    n = mib << 20
    return [("fastq", lambda: synth.fastq(n, seed=synth.SEED_FASTQ)),
            ("markov", lambda: synth.markov2(n, seed=synth.SEED_MARKOV)),
            ("wordtext", lambda: synth.wordtext(n, seed=synth.SEED_SERVE))]


def row(x: np.ndarray, mm, block_size: int, gpu: bool) -> dict:
    c = learned.encode(x, mm, block_size=block_size)
    e = aclz.aclz_acle_encode(c)
    blk, ll, ml, src, lits, bs, total = learned.read_tokens(c)
    m = ml > 0
    r = {"min_match": list(mm), "container_bytes": int(c.size), "acle_bytes": int(e.size),
         "ratio": round(x.size / e.size, 4), "est_ratio": round(x.size / learned.est_bytes(c), 4),
         "tokens": int(ll.size), "matches": int(m.sum()),
         "mean_match_len": round(float(ml[m].mean()), 2) if m.any() else 0.0}
    if gpu:
        for flat in (False, True):
            gbs, out = learned.decode_gbs(c, x.size, flatten=flat)
            if not np.array_equal(out.cpu().numpy(), x):
                raise RuntimeError("decode differs from the input")
            r["decode_gbs_flattened" if flat else "decode_gbs"] = round(gbs, 1)
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mib", type=int, default=64)
    ap.add_argument("--block-size", type=int, default=1 << 14)
    ap.add_argument("--gpu", action="store_true", help="also time the decode on the current GPU")
    ap.add_argument("--streams", default="fastq,markov,wordtext", help="comma-separated subset")
    ap.add_argument("--presets-only", action="store_true", help="skip the band sweep")
    args = ap.parse_args()
    want = set(args.streams.split(","))
    for name, make in streams(args.mib):
        if name not in want:
            continue
        x = make()
        for vname, mm in variants()[:3] if args.presets_only else variants():
            r = {"stream": name, "mib": args.mib, "block_size": args.block_size, "variant": vname}
            r.update(row(x, mm, args.block_size, args.gpu))
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
