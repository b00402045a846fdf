"""Encode throughput of the two greedy parsers that write the same
container: the host encoder (aclz_encode, all host cores) and the GPU parse
(aclz_encode_gpu, including the copies to and from the device).  The paper
places its encoder on the CPU and makes no speed claim for it (Sec. VI).

    python -m paper_2607_18541_gb300.encoders [--mib 256] [--presets base,tuned,pushed]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import aclz, synth

PRESETS = {"base": aclz.ACLZ_PRESET_BASE, "tuned": aclz.ACLZ_PRESET_TUNED, "pushed": aclz.ACLZ_PRESET_PUSH}


def streams(mib: int):
    n = mib << 20
    return [("fastq", lambda: synth.fastq(n, seed=synth.SEED_FASTQ)),
            ("markov", lambda: synth.markov2(n, seed=synth.SEED_MARKOV)),
            ("wordtext", lambda: synth.wordtext(n, seed=synth.SEED_SERVE))]


def run(mib: int, presets, block_size: int = 1 << 16, reps: int = 2):
    rows = []
    for name, make in streams(mib):
        x = make()
        for pr in presets:
            p = aclz.aclz_encode_params_default(PRESETS[pr])
            p.block_size = block_size
            aclz.aclz_encode_gpu(x[:1 << 20], p)  # warm the device and the kernels
            t = time.perf_counter()
            for _ in range(reps):
                c_host = aclz.aclz_encode(x, p)
            t_host = (time.perf_counter() - t) / reps
            t = time.perf_counter()
            for _ in range(reps):
                c_gpu = aclz.aclz_encode_gpu(x, p)
            t_gpu = (time.perf_counter() - t) / reps
            rows.append({"stream": name, "mib": mib, "preset": pr, "block_size": block_size,
                         "container_bytes": int(c_host.size), "identical": bool(np.array_equal(c_host, c_gpu)),
                         "host_mb_s": round(x.size / t_host / 1e6, 1), "host_threads": os.cpu_count(),
                         "gpu_mb_s": round(x.size / t_gpu / 1e6, 1)})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mib", type=int, default=256)
    ap.add_argument("--presets", default="base,tuned,pushed")
    a = ap.parse_args()
    for r in run(a.mib, a.presets.split(",")):
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
