"""Pure copy driven by a measured match-length distribution (the plateau
experiment of the limits section): the paper times its pure-copy harness
with the tuned match-length distribution of enwik9 instead of one length,
and reads the result (about 217 GB/s on H100) as the bandwidth limit at that
granularity.

Here the distribution comes from an encoded stream (word text, the enwik9
stand-in, at 12/16/24/32 by default): its match lengths form the table the
copy sweep draws each match length from (uniform random sources, geometric
literal runs of mean 4, as in the fixed-length sweep).  On a GPU the sweep
is decoded next to the stream itself and next to a fixed-length sweep at
the table's mean length, so the three numbers separate the length
distribution from everything else the real stream has (source locality,
copy chains, literal runs).

    python -m paper_2607_18541_gb300.plateau [--mib 256] [--sweep-mib 1024] [--gpu]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import learned, synth


def length_table(c) -> np.ndarray:
    """Match lengths of a container, in token order."""
    _, _, ml, _, _, _, _ = learned.read_tokens(c)
    return ml[ml > 0].astype(np.uint32)


def stats(sw: synth.CopySweep) -> dict:
    m = sw.match_len[sw.match_len > 0]
    return {"tokens": int(sw.n_tokens), "matches": int(m.size),
            "mean_match_len": round(float(m.mean()), 2) if m.size else 0.0,
            "match_bytes_fraction": round(float(m.sum()) / sw.total, 4)}


def _container(sw: synth.CopySweep):
    from . import aclz
    return aclz.aclz_pack(sw.total, sw.block_size, (4, 4, 4, 4), sw.blk_ntok, sw.lit_len, sw.match_len, sw.src,
                          sw.literals)


def run(mib: int, sweep_mib: int, block_size: int, mm, gpu: bool):
    x = synth.wordtext(mib << 20, seed=synth.SEED_SERVE)
    c = learned.encode(x, mm, block_size=block_size)
    table = length_table(c)
    rows = []
    real = {"what": "stream", "stream": f"wordtext_{mib}MiB", "min_match": list(mm), "matches": int(table.size),
            "mean_match_len": round(float(table.mean()), 2)}
    hist = synth.copy_sweep_lengths(sweep_mib << 20, block_size, table)
    mean_len = max(1, int(round(float(table.mean()))))
    fixed = synth.copy_sweep(sweep_mib << 20, block_size, mean_len)
    rows.append(real)
    rows.append({"what": "copy sweep, lengths drawn from the stream's", "mib": sweep_mib, **stats(hist)})
    rows.append({"what": f"copy sweep, fixed L = {mean_len}", "mib": sweep_mib, **stats(fixed)})
    if gpu:
        for r, cont, n, ref in ((rows[0], c, x.size, x), (rows[1], _container(hist), hist.total, None),
                                (rows[2], _container(fixed), fixed.total, None)):
            for flat in (False, True):
                gbs, out = learned.decode_gbs(cont, n, flatten=flat)
                if ref is not None and not np.array_equal(out.cpu().numpy(), ref):
                    raise RuntimeError("decode differs from the input")
                r["decode_gbs_flattened" if flat else "decode_gbs"] = round(gbs, 1)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mib", type=int, default=256, help="word text to take the length distribution from")
    ap.add_argument("--sweep-mib", type=int, default=1024)
    ap.add_argument("--block-size", type=int, default=1 << 16)
    ap.add_argument("--gpu", action="store_true")
    args = ap.parse_args()
    for r in run(args.mib, args.sweep_mib, args.block_size, (12, 16, 24, 32), args.gpu):
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
