"""Benchmark of the match-phase decode (output GB/s and fraction of the HBM
roofline) on the synthetic copy sweep: 1 GiB of output generated directly
as tokens, literal runs geometric (mean 4) of random bytes, matches of
fixed length L (default 1024) from sources uniform in [0, pos - L), decoded
with G-lane groups (Table II's experiment, Sec. III-C).

One JSON line on rank 0.  `value` is device-resident decode throughput
(container already in HBM); `e2e` is the same metric through the public C
ABI from pinned host buffers, the upload (host->device copy and index
build) and the read-back of the decoded bytes inside the timed region.
Beside the headline (at one GPU): `sweep`, the same recipe at the other
match lengths of Table II; `seek`, p50/p99 latency and GB/s of region seeks
served from a compressed word-text corpus held in HBM (the metric's second
half); `cpu_baseline`, the CPU oracle's sequential decoder on this same
workload.  `--impl reference` times that oracle decoder as the reference
arm (the same workload, or a bounded sample of it when K steps would take
over about two minutes).

Multi-GPU: the decode does not shard (absolute sources reach anywhere
earlier), so N ranks run N independent replicas (weak scaling, no
collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PAPER_H100 = {1024: 744, 512: 734, 256: 692, 128: 607, 64: 416, 32: 212}  # Table II, GB/s


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=1024)
    ap.add_argument("--total", type=int, default=1 << 30)
    ap.add_argument("--block-size", type=int, default=1 << 15)
    ap.add_argument("--G", type=int, default=32)
    ap.add_argument("--mode", default="auto", choices=["auto", "waves", "persistent"])
    ap.add_argument("--ctas-per-sm", type=int, default=2)
    ap.add_argument("--range-bytes", type=int, default=20480)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--sweep", default="32,64,128,256,512",
                    help="match lengths of the sweep block (same recipe; empty string: none)")
    ap.add_argument("--sweep-steps", type=int, default=20)
    ap.add_argument("--seek-gib", type=float, default=8.0,
                    help="serving corpus size for the seek block (0: no seek block)")
    ap.add_argument("--seek-requests", type=int, default=1000)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over the ranks of the process group (x itself alone)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(ms_max: float, bytes_per_rank: int, world: int) -> float:
    """Whole-job output GB/s of `world` independent replicas, each decoding
    bytes_per_rank per step, timed by the slowest rank."""
    return world * bytes_per_rank / (ms_max * 1e-3) / 1e9


def make_workload(total, bs, L, seed_offset=0):
    from paper_2607_18541_gb300 import synth
    return synth.copy_sweep(total, bs, L, seed=synth.SEED_COPY + L + seed_offset)


def algorithmic_bytes(sw) -> int:
    """16 B per token + literal bytes read + match source bytes read +
    output bytes written."""
    match_bytes = int(sw.match_len.astype(np.int64).sum())
    return 16 * sw.n_tokens + int(sw.literals.size) + match_bytes + int(sw.total)


def phase_bytes(sw, tags):
    """Algorithmic bytes of the two decode phases.  Wave 0: every token read,
    literals read and written, in-order matches read and written.  Deferred
    phase (waves >= 1): deferred match bytes read at the source and written
    at the target.  The two add up to algorithmic_bytes."""
    ml = sw.match_len.astype(np.int64)
    deferred = (np.asarray(tags) > 0) & (ml > 0)
    dbytes = int(ml[deferred].sum())
    w0 = 16 * sw.n_tokens + 2 * int(sw.literals.size) + 2 * (int(ml.sum()) - dbytes)
    return w0, 2 * dbytes, int(deferred.sum())


RATED_HBM_GBS = 7900.0  # GB300 HBM3e nominal bandwidth


def host_info() -> dict:
    """Core count and CPU model of the host running this process."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"host_cores": os.cpu_count(), "cpu_model": model}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_sources_sha() -> str:
    """Hash of the sources of the decode kernels (k_wave0, k_ranges and the
    copy helpers they inline): recorded traffic is valid only for these."""
    d = os.path.join(ROOT, "paper_2607_18541_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("aclz_decode.cu", "aclz_device.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary (profiles/traffic_k_ranges_<workload>.txt, lines "key: value"),
    if it was taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", f"traffic_k_ranges_{workload}.txt")
    if not os.path.exists(p):
        return None
    d = {}
    with open(p) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                d[k.strip()] = v.strip()
    if d.get("kernel_sources_sha") != kernel_sources_sha():
        return None
    try:
        return int(d["dram_bytes_read"]) + int(d["dram_bytes_write"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
                power.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def cpu_baseline(args, seconds: float):
    """The oracle's sequential decoder (one host thread) on the benchmark's
    own workload (the same generated container), decoded repeatedly for
    about `seconds`."""
    import oracle
    sw = make_workload(args.total, args.block_size, args.L)
    c = oracle.pack_sweep(sw, tags=False)
    oracle.decode(c)  # warm
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.decode(c)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    gbs = n * args.total / el / 1e9
    return {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", **host_info(),
            "sample": f"the benchmark workload ({args.total >> 20} MiB copy sweep, L={args.L}), decoded {n} "
                      f"times in {el:.1f} s by the sequential oracle decoder on one host thread"}


def run_reference(args):
    """The oracle's sequential decoder as the reference arm: W warm-up and K
    timed decodes of a bounded sample of the same workload (a copy sweep of
    the same recipe, at most 128 MiB, shrunk so K decodes take <= ~2 min)."""
    import oracle
    rank, world, local = dist_env()
    if rank != 0:
        return
    sample = args.total
    sw = make_workload(sample, args.block_size, args.L)
    c = oracle.pack_sweep(sw, tags=False)
    t0 = time.perf_counter()
    for _ in range(max(1, args.warmup)):
        oracle.decode(c)
    per = (time.perf_counter() - t0) / max(1, args.warmup)
    if per * args.steps > 120.0:
        # a bounded sample of the same recipe, so K steps take about 2 min
        sample = max(1 << 20, int(sample * 120.0 / (per * args.steps)) & ~((1 << 20) - 1))
        sw = make_workload(sample, args.block_size, args.L, seed_offset=1)
        c = oracle.pack_sweep(sw, tags=False)
        oracle.decode(c)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.decode(c)
    el = time.perf_counter() - t0
    gbs = args.steps * sample / el / 1e9
    cb = {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", **host_info(),
          "sample": f"{sample >> 20} MiB copy sweep (L={args.L}, same recipe"
                    f"{'' if sample == args.total else ', a bounded sample of the workload'}) per step, "
                    f"{args.steps} steps in {el:.1f} s, sequential oracle decoder on one host thread"}
    line = {
        "impl": "reference",
        "metric": f"match-phase decode output GB/s (copy sweep, L={args.L})",
        "value": cb["value"], "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic",
        "config": workload_config(args, {"same_config": sample == args.total}),
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, extra):
    cfg = {"workload": f"copy_sweep_{args.total >> 20}MiB_L{args.L}", "total_bytes": args.total,
           "match_len": args.L, "lit_mean": 4, "block_size": args.block_size, "G": args.G,
           "mode": args.mode, "ctas_per_sm": args.ctas_per_sm, "range_bytes": args.range_bytes,
           "lanes": args.G * ((args.total + args.block_size - 1) // args.block_size),
           "l2": "flushed between timed steps (256 MiB write)" if not args.no_flush else "not flushed"}
    if extra:
        cfg.update(extra)
    return cfg


MODE = {"auto": 2, "waves": 0, "persistent": 1}
LIB_RANGE_BYTES = 20480  # the work-range size an upload picks
KERNEL = {0: "k_wave_copy (one launch per wave >= 1)", 1: "k_ranges (persistent, deferred matches)"}


def sweep_leg(args, dev, st, peak):
    """Table II's experiment over the match length: the same 1 GiB recipe at
    each L of --sweep, decoded in the library's automatic mode (per-wave
    kernels for short matches, the persistent staged schedule for long
    ones), CUDA-event timed with the L2 flushed between steps."""
    import torch
    from paper_2607_18541_gb300 import aclz
    Ls = [int(v) for v in args.sweep.split(",") if v.strip()]
    rows = []
    if not Ls:
        return rows
    out = torch.empty(((args.total + 15) // 16) * 16, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for L in Ls:
        sw = make_workload(args.total, args.block_size, L)
        c = aclz.aclz_pack(sw.total, sw.block_size, (4, 4, 4, 4), sw.blk_ntok, sw.lit_len, sw.match_len,
                           sw.src, sw.literals)
        h = aclz.aclz_upload(c, st)
        try:
            if args.range_bytes != LIB_RANGE_BYTES:
                aclz.aclz_set_range_bytes(h, args.range_bytes, st)
            info = aclz.aclz_handle_info(h)
            cfg = dict(G=args.G, mode=MODE["auto"], ctas_per_sm=args.ctas_per_sm)
            plan, launches = aclz.aclz_decode_plan(h, **cfg)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.sweep_steps)]
            with torch.cuda.stream(st):
                for _ in range(3):
                    aclz.aclz_decode_all(h, out, stream=st, **cfg)
                for i, (a, b) in enumerate(ev):
                    if not args.no_flush:
                        flush.fill_(i & 0xff)
                    a.record(st)
                    aclz.aclz_decode_all(h, out, stream=st, **cfg)
                    b.record(st)
                st.synchronize()
            assert aclz.aclz_device_status(h, st) == 0
            ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
            abytes = algorithmic_bytes(sw)
            rows.append({"L": L, "value": round(sw.total / (ms * 1e-3) / 1e9, 1), "unit": "GB/s",
                         "ms_per_step": round(ms, 4), "step_frac": round(abytes / (ms * 1e-3) / 1e9 / peak, 4),
                         "algorithmic_bytes_per_step": abytes, "mode": "persistent" if plan["mode"] == 1 else "waves",
                         "n_waves": info.n_waves, "launches_per_step": launches,
                         "paper_h100_context": PAPER_H100.get(L)})
        finally:
            aclz.aclz_free(h)
    del out, flush
    return rows


def seek_leg(args, dev):
    """The serving configuration: order-3 Markov word text (50k-word Zipf
    vocabulary) of --seek-gib GiB, encoded at 12/16/24/32 in 64 KiB blocks,
    held compressed in HBM; region seeks of log-uniform 16 KiB-256 MiB at
    Poisson arrivals (25/50/75/90% of the saturated rate), admitted by free
    HBM and served by the continuous-batching loop.  Every saturated-run
    result is then compared on the device with the corpus slice it names."""
    import torch
    from paper_2607_18541_gb300 import aclz, serve, synth
    total = int(args.seek_gib * (1 << 30))
    t0 = time.perf_counter()
    x, c = serve.build_corpus(total, chain_depth=4)
    t_build = time.perf_counter() - t0
    st = torch.cuda.current_stream()
    t0 = time.perf_counter()
    h = aclz.aclz_upload(c, st, flags=aclz.ACLZ_UPLOAD_FLATTEN)
    t_up = time.perf_counter() - t0
    try:
        rows = serve.serve_benchmark(h, total, args.seek_requests)
        # every result of the saturated request set against the corpus
        xd = torch.from_numpy(x).to(dev)
        del x
        lo, hi = 16 << 10, min(256 << 20, total)
        _, starts, sizes = synth.requests(args.seek_requests, 1.0, lo, hi, total, synth.SEED_SERVE + 7)
        bad = []

        def check(i, buf):
            a, n = int(starts[i]), int(sizes[i])
            if not torch.equal(buf[:n], xd[a:a + n]):
                bad.append(i)

        free, _ = torch.cuda.mem_get_info()
        srv = serve.Server(h, int(free * 0.5))
        srv.run(np.zeros(args.seek_requests), starts, sizes, on_done=check)
        assert aclz.aclz_device_status(h, st) == 0
        del xd
    finally:
        aclz.aclz_free(h)
    sat = rows[0]
    loads = [r for r in rows[1:]]
    p50 = max(r["p50_ms"] for r in loads) if loads else sat["p50_ms"]
    return {"workload": f"serve_wordtext_{args.seek_gib:g}GiB_64KiB_blocks",
            "corpus_bytes": total, "container_bytes": int(c.size), "block_size": 1 << 16,
            "thresholds": "12/16/24/32", "request_sizes": "log-uniform 16 KiB-256 MiB",
            "requests_per_load": args.seek_requests, "saturated_gbs": sat["gbs"],
            "p50_ms": {str(r["load"]): r["p50_ms"] for r in rows},
            "p99_ms": {str(r["load"]): r["p99_ms"] for r in rows},
            "gbs": {str(r["load"]): r["gbs"] for r in rows},
            "clock_bias_ms_max": max(r["clock_bias_ms"] for r in rows),
            "verified_requests": args.seek_requests - len(bad), "mismatched_requests": len(bad),
            "corpus_build_s": round(t_build, 1), "upload_s": round(t_up, 2),
            "latency": "GPU completion event minus Poisson arrival (host clock), per request"}


def run_ours(args):
    import torch
    from paper_2607_18541_gb300 import aclz

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    aclz.lib()
    sw = make_workload(args.total, args.block_size, args.L, seed_offset=0)
    c = aclz.aclz_pack(sw.total, sw.block_size, (4, 4, 4, 4), sw.blk_ntok, sw.lit_len, sw.match_len,
                       sw.src, sw.literals)
    abytes = algorithmic_bytes(sw)
    st = torch.cuda.Stream(device=dev)
    h = aclz.aclz_upload(c, st)
    if args.range_bytes != LIB_RANGE_BYTES:
        aclz.aclz_set_range_bytes(h, args.range_bytes, st)
    info = aclz.aclz_handle_info(h)
    cfg = dict(G=args.G, mode=MODE[args.mode], ctas_per_sm=args.ctas_per_sm)
    plan, launches_per_step = aclz.aclz_decode_plan(h, **cfg)
    w0_bytes, def_bytes, n_def = phase_bytes(sw, aclz.aclz_tags(h))
    out = torch.empty(((sw.total + 15) // 16) * 16, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    with torch.cuda.stream(st):
        for ev in mids:
            ev.record(st)  # creates the CUDA event the library records into
        for _ in range(args.warmup):
            aclz.aclz_decode_all(h, out, stream=st, **cfg)
        st.synchronize()
        assert aclz.aclz_device_status(h, st) == 0
        clk = ClockSampler(local)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk.start()
        time.sleep(0.2)
        t_wall0 = time.perf_counter()
        for i in range(args.steps):
            if not args.no_flush:
                flush.fill_(i & 0xff)
            starts[i].record(st)
            aclz.aclz_decode_all_ev(h, out, mids[i], stream=st, **cfg)
            ends[i].record(st)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        clocks = clk.stop()
        if world > 1:
            torch.distributed.barrier()
    assert aclz.aclz_device_status(h, st) == 0
    ms = [s_.elapsed_time(e) for s_, e in zip(starts, ends)]
    ms_w0 = [s_.elapsed_time(m) for s_, m in zip(starts, mids)]
    ms_def = [m.elapsed_time(e) for m, e in zip(mids, ends)]
    ms_step = sum(ms) / len(ms)
    ms_max = max_over_ranks(ms_step, dev)
    value = replica_value(ms_max, sw.total, world)
    peak, peak_kind = peaks()
    w0_ms, d_ms = statistics.mean(ms_w0), statistics.mean(ms_def)
    if d_ms >= w0_ms and n_def:
        kern, kbytes, kms = KERNEL[plan["mode"]], def_bytes, d_ms
        klaunch = launches_per_step - 1
    else:
        kern, kbytes, kms = "k_wave0 (tokens, literals, in-order matches)", w0_bytes, w0_ms
        klaunch = 1
    achieved = kbytes / (kms * 1e-3) / 1e9
    workload = workload_config(args, None)["workload"]
    traffic = recorded_traffic(workload)

    # end to end through the C ABI from pinned host memory: the container as
    # written once with its wave tags (aclz_export), so each upload checks
    # them in parallel instead of computing them block after block
    c_tagged = aclz.aclz_export(h)
    host_c = torch.from_numpy(c_tagged).pin_memory()
    host_out = torch.empty(sw.total, dtype=torch.uint8).pin_memory()
    def e2e_steps(container, steps):
        ms, up = [], []
        with torch.cuda.stream(st):
            for i in range(steps + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                hh = aclz.aclz_upload(container, st)
                if args.range_bytes != LIB_RANGE_BYTES:
                    aclz.aclz_set_range_bytes(hh, args.range_bytes, st)
                t1 = time.perf_counter()
                aclz.aclz_decode_all(hh, out, stream=st, **cfg)
                host_out.copy_(out[:sw.total], non_blocking=True)
                st.synchronize()
                dt = time.perf_counter() - t0
                aclz.aclz_free(hh)
                if i:
                    ms.append(dt * 1e3)
                    up.append((t1 - t0) * 1e3)
        # medians: one host-side stall (page cache, scheduler) in a handful
        # of steps would otherwise decide the figure
        return statistics.median(ms), statistics.median(up)

    e2e_mean, e2e_up = e2e_steps(host_c.numpy(), args.e2e_steps)
    e2e_val = replica_value(max_over_ranks(e2e_mean, dev), sw.total, world)
    # the same through an upload of the untagged container, whose minimal
    # wave tags the upload computes (an ordered pass over the blocks)
    host_u = torch.from_numpy(c).pin_memory()
    ut_mean, ut_up = e2e_steps(host_u.numpy(), args.e2e_steps)
    ut_val = replica_value(max_over_ranks(ut_mean, dev), sw.total, world)
    if rank == 0:
        line = {
            "metric": f"match-phase decode output GB/s (copy sweep, L={args.L})",
            "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(args, {"n_waves": info.n_waves, "n_tokens": info.n_tokens,
                                             "n_deferred": info.n_deferred, "resolved": plan,
                                             "algorithmic_bytes_per_step": abytes}),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kern,
                         "achieved_is": "algorithmic bytes of the kernel per launch / its CUDA-event time",
                         "rated_peak": RATED_HBM_GBS, "frac_of_rated": round(achieved / RATED_HBM_GBS, 4),
                         "launches_per_step": klaunch, "algorithmic_bytes_per_step": kbytes,
                         "ms_per_step": round(kms, 5), "peak_kind": f"{peak_kind} copy (burst)"},
            "phases": {"wave0_ms": round(w0_ms, 5), "wave0_bytes": w0_bytes,
                       "deferred_ms": round(d_ms, 5), "deferred_bytes": def_bytes,
                       "step_achieved_gbs": round(abytes / (ms_step * 1e-3) / 1e9, 1),
                       "step_frac": round(abytes / (ms_step * 1e-3) / 1e9 / peak, 4)},
            "clocks": clocks,
            "gpu_launches": launches_per_step * args.steps,
            "e2e": {"value": round(e2e_val, 2), "unit": "GB/s", "h2d_bytes_per_step": int(c_tagged.size),
                    "d2h_bytes_per_step": int(sw.total), "steps": args.e2e_steps,
                    "ms_per_step": round(e2e_mean, 3), "upload_ms": round(e2e_up, 3), "stat": "median of steps",
                    "includes": "upload of the tagged container (copy, validation, tag check, worklists), "
                                "decode, read-back of the output",
                    "untagged_upload": {"value": round(ut_val, 2), "unit": "GB/s", "ms_per_step": round(ut_mean, 3),
                                        "upload_ms": round(ut_up, 3), "h2d_bytes_per_step": int(c.size),
                                        "includes": "upload of the container without wave tags (the upload "
                                                    "computes minimal tags), decode, read-back"}},
            "paper_h100_context": {"value": PAPER_H100.get(args.L), "unit": "GB/s",
                                   "what": "purecopy.cu synthetic copy, 1 GB, H100 (Table II)"},
            "wall_s_timed": round(t_wall, 3),
        }
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(args, args.cpu_seconds)
            if args.sweep.strip():
                line["sweep"] = sweep_leg(args, dev, st, peak)
            if args.seek_gib > 0:
                line["seek"] = seek_leg(args, dev)
        print(json.dumps(line), flush=True)
    aclz.aclz_free(h)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
