"""Seeded synthetic inputs shared by the CPU oracle and the GPU library.

The generators live in ``synth.c`` (compiled to ``libaclz_synth.so`` beside
it) and hold none of the codec's arithmetic: they produce byte streams to be
compressed, directly generated copy-sweep token arrays, stream sizes for the
batched workload and request traces for the serving loop.  Every draw comes
from xoshiro256** seeded by splitmix64, so the same seed gives the same bytes
on every machine.

Workload recipes (the paper's datasets are absent; these stand in for them):

* ``markov2``: order-2 Markov bytes over 0x30..0x6F, per-context
  Dirichlet(0.3) next-symbol laws, 5% of positions start a verbatim repeat of
  geometric length (mean 12) from a uniform earlier position (stand-in for the
  Silesia-style mixed corpora of Sec. III-B).
* ``copy_sweep``: the synthetic copy experiment of Table II: literal runs
  geometric (mean 4) of random bytes, matches of fixed length L from sources
  uniform in [0, pos - L).
* ``fastq``: FASTQ-like records (stand-in for the NA12878/ERR194147 FASTQ of
  Sec. II): 150-base reads from a 4.6 Mbase random reference with 1%
  substitutions and 0.1% N, Phred+33 qualities from a drifting order-1 chain
  over 38 levels.
* ``wordtext``: order-3 Markov word text over a 50k-word Zipf(1.1)
  vocabulary (stand-in for enwik9-like text).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_SO = os.path.join(_HERE, "libaclz_synth.so")
_lock = threading.Lock()
_lib = None

# fixed seeds of the five workloads
SEED_MARKOV = 0xACE00001
SEED_COPY = 0xACE00002
SEED_FASTQ = 0xACE00003
SEED_BATCH = 0xACE00004
SEED_SERVE = 0xACE00005


def build(force: bool = False) -> str:
    """Compile the generator library with gcc (no FP contraction, so the
    output is identical on x86-64 and AArch64)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            dp = ctypes.POINTER(ctypes.c_double)
            L.synth_markov2.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_double]
            L.synth_markov2.restype = ctypes.c_int
            L.synth_markov_model_new.argtypes = [ctypes.c_uint64, ctypes.c_double]
            L.synth_markov_model_new.restype = ctypes.c_void_p
            L.synth_markov_model_free.argtypes = [ctypes.c_void_p]
            L.synth_markov_model_free.restype = None
            L.synth_markov2_gen.argtypes = [ctypes.c_void_p, u8p, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_uint32, ctypes.c_uint32]
            L.synth_markov2_gen.restype = ctypes.c_int
            L.synth_fastq.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
            L.synth_fastq.restype = ctypes.c_int
            L.synth_wordtext.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            L.synth_wordtext.restype = ctypes.c_int
            L.synth_vocab_new.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double]
            L.synth_vocab_new.restype = ctypes.c_void_p
            L.synth_vocab_free.argtypes = [ctypes.c_void_p]
            L.synth_vocab_free.restype = None
            L.synth_wordtext_chunk.argtypes = [ctypes.c_void_p, u8p, ctypes.c_uint64,
                                               ctypes.c_uint64, ctypes.c_uint64]
            L.synth_wordtext_chunk.restype = ctypes.c_int
            L.synth_copy_sweep.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u32p, u64p,
                                           ctypes.c_uint64, u8p, ctypes.c_uint64, u64p]
            L.synth_copy_sweep.restype = ctypes.c_int64
            L.synth_copy_sweep_lengths.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u32p, ctypes.c_uint64,
                                                   ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u32p, u64p,
                                                   ctypes.c_uint64, u8p, ctypes.c_uint64, u64p]
            L.synth_copy_sweep_lengths.restype = ctypes.c_int64
            L.synth_stream_sizes.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_uint64, u64p, u64p]
            L.synth_stream_sizes.restype = ctypes.c_int
            L.synth_requests.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, dp,
                                         u64p, u64p]
            L.synth_requests.restype = ctypes.c_int
            L.synth_rng_sequence.argtypes = [ctypes.c_uint64, u64p, ctypes.c_uint64]
            L.synth_rng_sequence.restype = ctypes.c_uint64
            L.synth_ln.argtypes = [ctypes.c_double]
            L.synth_ln.restype = ctypes.c_double
            L.synth_exp.argtypes = [ctypes.c_double]
            L.synth_exp.restype = ctypes.c_double
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc: int, what: str) -> None:
    if rc < 0:
        raise RuntimeError(f"synth.{what} failed with code {rc}")


def rng_sequence(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    lib().synth_rng_sequence(seed, _ptr(out, ctypes.c_uint64), n)
    return out


def markov2(n: int, seed: int = SEED_MARKOV, repeat_every: int = 20, repeat_mean: int = 12,
            alpha: float = 0.3, out: np.ndarray | None = None) -> np.ndarray:
    """Order-2 Markov bytes; ``repeat_every=20`` is the 5% repeat rate."""
    buf = np.empty(n, dtype=np.uint8) if out is None else out
    _check(lib().synth_markov2(_ptr(buf, ctypes.c_uint8), n, seed, repeat_every, repeat_mean,
                               alpha), "markov2")
    return buf


class MarkovModel:
    """A reusable order-2 Markov model (its Dirichlet draws are the slow part),
    so many streams can be drawn from one model in parallel threads."""

    def __init__(self, model_seed: int = SEED_BATCH, alpha: float = 0.3):
        self._h = lib().synth_markov_model_new(model_seed, alpha)
        if not self._h:
            raise MemoryError("synth Markov model")

    def generate(self, n: int, seed: int, repeat_every: int = 20, repeat_mean: int = 12,
                 out: np.ndarray | None = None) -> np.ndarray:
        buf = np.empty(n, dtype=np.uint8) if out is None else out
        _check(lib().synth_markov2_gen(self._h, _ptr(buf, ctypes.c_uint8), n, seed, repeat_every,
                                       repeat_mean), "markov2_gen")
        return buf

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            lib().synth_markov_model_free(h)


def fastq(n: int, seed: int = SEED_FASTQ, out: np.ndarray | None = None) -> np.ndarray:
    buf = np.empty(n, dtype=np.uint8) if out is None else out
    _check(lib().synth_fastq(_ptr(buf, ctypes.c_uint8), n, seed), "fastq")
    return buf


def wordtext(n: int, seed: int = SEED_SERVE, chunk_bytes: int = 64 << 20, threads: int = 0,
             out: np.ndarray | None = None) -> np.ndarray:
    """Order-3 Markov word text of exactly n bytes, generated in independent
    chunks of ``chunk_bytes`` (in parallel when ``threads`` > 1)."""
    buf = np.empty(n, dtype=np.uint8) if out is None else out
    L = lib()
    threads = threads or min(16, os.cpu_count() or 1)
    vocab = L.synth_vocab_new(seed, 50000, 1.1)
    if not vocab:
        raise MemoryError("synth vocabulary")
    try:
        nchunks = (n + chunk_bytes - 1) // chunk_bytes
        base = buf.ctypes.data

        def work(c: int) -> None:
            lo = c * chunk_bytes
            ln = min(chunk_bytes, n - lo)
            rc = L.synth_wordtext_chunk(vocab, ctypes.cast(base + lo, ctypes.POINTER(ctypes.c_uint8)),
                                        ln, seed, c)
            _check(rc, "wordtext")

        if threads > 1 and nchunks > 1:
            from concurrent.futures import ThreadPoolExecutor
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(work, range(nchunks)))
        else:
            for c in range(nchunks):
                work(c)
    finally:
        L.synth_vocab_free(vocab)
    return buf


class CopySweep:
    """Directly generated token arrays of the synthetic copy sweep."""

    def __init__(self, total: int, block_size: int, L: int, lit_mean: int, seed: int,
                 blk_ntok: np.ndarray, lit_len: np.ndarray, match_len: np.ndarray,
                 src: np.ndarray, literals: np.ndarray):
        self.total, self.block_size, self.L, self.lit_mean, self.seed = total, block_size, L, lit_mean, seed
        self.blk_ntok, self.lit_len, self.match_len, self.src = blk_ntok, lit_len, match_len, src
        self.literals = literals

    @property
    def n_tokens(self) -> int:
        return int(self.lit_len.shape[0])


def copy_sweep(total: int, block_size: int, L: int, lit_mean: int = 4,
               seed: int = SEED_COPY) -> CopySweep:
    nb = (total + block_size - 1) // block_size
    cap = total // max(1, L) + nb + 1
    blk = np.zeros(nb, dtype=np.uint32)
    ll = np.empty(cap, dtype=np.uint32)
    ml = np.empty(cap, dtype=np.uint32)
    sr = np.empty(cap, dtype=np.uint64)
    lits = np.empty(max(total, 1), dtype=np.uint8)
    nlit = np.zeros(1, dtype=np.uint64)
    nt = lib().synth_copy_sweep(total, block_size, L, lit_mean, seed, _ptr(blk, ctypes.c_uint32),
                                _ptr(ll, ctypes.c_uint32), _ptr(ml, ctypes.c_uint32),
                                _ptr(sr, ctypes.c_uint64), cap, _ptr(lits, ctypes.c_uint8), total,
                                _ptr(nlit, ctypes.c_uint64))
    _check(int(nt), "copy_sweep")
    nt = int(nt)
    return CopySweep(total, block_size, L, lit_mean, seed, blk, ll[:nt].copy(), ml[:nt].copy(),
                     sr[:nt].copy(), lits[:int(nlit[0])].copy())


def copy_sweep_lengths(total: int, block_size: int, lengths, lit_mean: int = 4,
                       seed: int = SEED_COPY) -> CopySweep:
    """The copy sweep with every match length drawn uniformly from
    `lengths` (e.g. the match lengths of an encoded stream: its empirical
    distribution) instead of one fixed L."""
    table = np.ascontiguousarray(lengths, dtype=np.uint32)
    if table.size == 0 or int(table.min()) == 0:
        raise ValueError("lengths must be non-empty and positive")
    nb = (total + block_size - 1) // block_size
    cap = total // int(table.min()) + nb + 1
    blk = np.zeros(nb, dtype=np.uint32)
    ll = np.empty(cap, dtype=np.uint32)
    ml = np.empty(cap, dtype=np.uint32)
    sr = np.empty(cap, dtype=np.uint64)
    lits = np.empty(max(total, 1), dtype=np.uint8)
    nlit = np.zeros(1, dtype=np.uint64)
    nt = lib().synth_copy_sweep_lengths(total, block_size, _ptr(table, ctypes.c_uint32), table.size, lit_mean,
                                        seed, _ptr(blk, ctypes.c_uint32), _ptr(ll, ctypes.c_uint32),
                                        _ptr(ml, ctypes.c_uint32), _ptr(sr, ctypes.c_uint64), cap,
                                        _ptr(lits, ctypes.c_uint8), total, _ptr(nlit, ctypes.c_uint64))
    _check(int(nt), "copy_sweep_lengths")
    nt = int(nt)
    return CopySweep(total, block_size, 0, lit_mean, seed, blk, ll[:nt].copy(), ml[:nt].copy(),
                     sr[:nt].copy(), lits[:int(nlit[0])].copy())


def stream_sizes(n: int, lo: int, hi: int, seed: int = SEED_BATCH):
    sizes = np.empty(n, dtype=np.uint64)
    seeds = np.empty(n, dtype=np.uint64)
    _check(lib().synth_stream_sizes(n, lo, hi, seed, _ptr(sizes, ctypes.c_uint64),
                                    _ptr(seeds, ctypes.c_uint64)), "stream_sizes")
    return sizes, seeds


def batch_stream(i: int, size: int, seed: int, model: MarkovModel | None = None) -> np.ndarray:
    """Stream i of the batched workload: even index Markov bytes (from one
    shared model, per-stream sequence seed), odd index FASTQ-like text."""
    if i % 2 == 0:
        return (model or MarkovModel()).generate(size, seed)
    return fastq(size, seed)


def requests(n: int, rate_per_s: float, lo: int, hi: int, corpus: int, seed: int = SEED_SERVE + 7):
    arr = np.empty(n, dtype=np.float64)
    st = np.empty(n, dtype=np.uint64)
    sz = np.empty(n, dtype=np.uint64)
    _check(lib().synth_requests(n, rate_per_s, lo, hi, corpus, seed, _ptr(arr, ctypes.c_double),
                                _ptr(st, ctypes.c_uint64), _ptr(sz, ctypes.c_uint64)), "requests")
    return arr, st, sz
