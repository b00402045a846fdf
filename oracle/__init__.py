"""CPU oracle for absolute-offset LZ77 decode (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it; the only module both sides use is the seeded input
generator ``paper_2607_18541_gb300.synth``.

``aclz_oracle.c`` holds the plain sequential definitions (greedy exact-prefix
chain encoder with distance-class minimum match lengths, Sec. IV-B; the
sequential decoder; minimal wave tags; validation; chunked FNV-1a; the
order-0 tile entropy estimate); ``ans.c`` the tile entropy layer (order-0
rANS over 64 KiB tiles and the ACLE container of a v1 container's token byte
planes and literals).  This module wraps both with ctypes and adds
pure-Python brute-force references used to pin them on tiny inputs.

Parity status: every function here is pinned by tests in
``tests/test_oracle.py`` (published FNV vectors, closed forms, brute force,
round trips, invariants) and ``tests/test_ans_oracle.py`` (frequency rule
by hand, closed-form word counts, code-length bounds, round trips), except
``est_bytes`` beyond its closed-form cases, whose absolute scale is a
reading of the paper, not something it prints.
"""
from __future__ import annotations

import ctypes
import os
import struct
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aclz_oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "ans.c"))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, E_INVAL, E_CORRUPT, E_NOMEM, E_CAPACITY = 0, -1, -2, -3, -4
DIST_BOUNDS = (128, 16384, 2097152)          # Sec. IV-B distance bands
PRESET_BASE = (6, 8, 10, 12)                 # Sec. IV-B
PRESET_TUNED = (12, 16, 24, 32)              # Sec. IV-B
PRESET_PUSH = (16, 24, 32, 48)               # Sec. IV-C
FNV_BASIS = 14695981039346656037
FNV_PRIME = 1099511628211
UNLIMITED_DEPTH = 0xFFFFFFFF
UNLIMITED_WINDOW = (1 << 64) - 1


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(map(os.path.getmtime, _SRCS)):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"])
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
            c_u64, c_u32 = ctypes.c_uint64, ctypes.c_uint32
            L.oracle_decode.argtypes = [u8p, c_u64, u8p, c_u64]
            L.oracle_validate.argtypes = [u8p, c_u64]
            L.oracle_min_tags.argtypes = [u8p, c_u64, u32p, u32p]
            L.oracle_retag.argtypes = [u8p, c_u64, u32p]
            L.oracle_strip_tags.argtypes = [u8p, c_u64]
            L.oracle_container_bytes.argtypes = [c_u64, c_u32, c_u64, c_u64]
            L.oracle_container_bytes.restype = c_u64
            L.oracle_pack.argtypes = [c_u64, c_u32, u8p, u32p, u32p, u32p, u64p, c_u64, u8p, c_u64,
                                      u8p, c_u64, ctypes.c_int]
            L.oracle_pack.restype = ctypes.c_int64
            L.oracle_encode.argtypes = [u8p, c_u64, c_u32, u8p, u8p, c_u32, c_u64, u8p, c_u64]
            L.oracle_encode.restype = ctypes.c_int64
            L.oracle_encode_bound.argtypes = [c_u64, c_u32]
            L.oracle_encode_bound.restype = c_u64
            L.oracle_check_thresholds.argtypes = [u8p, c_u64]
            L.oracle_fnv1a64.argtypes = [u8p, c_u64, c_u64]
            L.oracle_fnv1a64.restype = c_u64
            L.oracle_fnv_chunked.argtypes = [u8p, c_u64]
            L.oracle_fnv_chunked.restype = c_u64
            L.oracle_est_bytes.argtypes = [u8p, c_u64, ctypes.POINTER(ctypes.c_double)]
            L.oracle_stats.argtypes = [u8p, c_u64, u64p]
            L.oracle_ans_quantize.argtypes = [u64p, c_u64, ctypes.POINTER(ctypes.c_uint16)]
            L.oracle_ans_tile_bound.argtypes = [c_u64]
            L.oracle_ans_tile_bound.restype = c_u64
            L.oracle_ans_encode_tile.argtypes = [u8p, c_u32, u8p, c_u64, u64p]
            L.oracle_ans_decode_tile.argtypes = [u8p, c_u64, u8p, c_u32]
            L.oracle_acle_bound.argtypes = [u8p, c_u64, u64p]
            L.oracle_acle_encode.argtypes = [u8p, c_u64, u8p, c_u64, u64p]
            L.oracle_acle_decoded_size.argtypes = [u8p, c_u64]
            L.oracle_acle_decoded_size.restype = c_u64
            L.oracle_acle_decode.argtypes = [u8p, c_u64, u8p, c_u64]
            _lib = L
    return _lib


def _u8(a) -> ctypes.POINTER(ctypes.c_uint8):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _arr(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    return np.ascontiguousarray(x, dtype=np.uint8)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle.{what}: code {code}")
        self.code = code


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise OracleError(int(rc), what)
    return rc


# ------------------------------------------------------------------ encode

def encode(x, block_size: int, mm=PRESET_BASE, block_mm=None, chain_depth: int = 64,
           window: int = UNLIMITED_WINDOW) -> np.ndarray:
    """Greedy exact-prefix chain encoder; returns the container bytes with
    minimal wave tags."""
    x = _arr(x)
    n = int(x.size)
    cap = int(lib().oracle_encode_bound(n, block_size))
    out = np.empty(cap, dtype=np.uint8)
    mma = np.array(mm, dtype=np.uint8)
    bmm = None if block_mm is None else np.ascontiguousarray(block_mm, dtype=np.uint8).reshape(-1)
    rc = lib().oracle_encode(_u8(x), n, block_size, _u8(mma), None if bmm is None else _u8(bmm),
                             chain_depth, window, _u8(out), cap)
    size = _check(int(rc), "encode")
    return out[:size].copy()


def pack(total_len: int, block_size: int, blk_ntok, lit_len, match_len, src, literals,
         mm=(4, 4, 4, 4), tags: bool = True) -> np.ndarray:
    """Container from token arrays, with minimal wave tags unless tags=False."""
    blk = np.ascontiguousarray(blk_ntok, dtype=np.uint32)
    ll = np.ascontiguousarray(lit_len, dtype=np.uint32)
    ml = np.ascontiguousarray(match_len, dtype=np.uint32)
    sr = np.ascontiguousarray(src, dtype=np.uint64)
    lits = _arr(literals) if len(literals) else np.zeros(1, dtype=np.uint8)
    nl = len(literals)
    cap = int(lib().oracle_container_bytes(total_len, block_size, ll.size, nl))
    out = np.empty(cap, dtype=np.uint8)
    mma = np.array(mm, dtype=np.uint8)
    rc = lib().oracle_pack(total_len, block_size, _u8(mma), blk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                           ll.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                           ml.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                           sr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ll.size, _u8(lits), nl,
                           _u8(out), cap, 1 if tags else 0)
    size = _check(int(rc), "pack")
    return out[:size].copy()


def pack_sweep(sweep, tags: bool = True) -> np.ndarray:
    """Container of a generated copy sweep (``synth.copy_sweep``)."""
    return pack(sweep.total, sweep.block_size, sweep.blk_ntok, sweep.lit_len, sweep.match_len,
                sweep.src, sweep.literals, tags=tags)


# ------------------------------------------------------------------ decode

def decode(c) -> np.ndarray:
    c = _arr(c)
    info = header(c)
    out = np.empty(max(1, info.total_len), dtype=np.uint8)
    _check(lib().oracle_decode(_u8(c), c.size, _u8(out), out.size), "decode")
    return out[:info.total_len]


def decode_range(c, lo: int, hi: int) -> np.ndarray:
    """out[lo:hi] of the sequential decode (the definition of a range read)."""
    full = decode(c)
    if not (0 <= lo <= hi <= full.size):
        raise OracleError(E_INVAL, "decode_range")
    return full[lo:hi].copy()


def validate(c) -> int:
    c = _arr(c)
    return int(lib().oracle_validate(_u8(c), c.size))


def check_thresholds(c) -> int:
    c = _arr(c)
    return int(lib().oracle_check_thresholds(_u8(c), c.size))


def min_tags(c):
    c = _arr(c)
    info = header(c)
    tags = np.zeros(max(1, info.n_tokens), dtype=np.uint32)
    nw = ctypes.c_uint32(0)
    _check(lib().oracle_min_tags(_u8(c), c.size, tags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                 ctypes.byref(nw)), "min_tags")
    return tags[:info.n_tokens], int(nw.value)


def retag(c, extra=None) -> np.ndarray:
    """Copy of c with tags = minimal requirement + extra (legal, non-minimal)."""
    c = _arr(c).copy()
    ex = None
    if extra is not None:
        ex = np.ascontiguousarray(extra, dtype=np.uint32)
    _check(lib().oracle_retag(_u8(c), c.size,
                              None if ex is None else ex.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))),
           "retag")
    return c


def strip_tags(c) -> np.ndarray:
    c = _arr(c).copy()
    _check(lib().oracle_strip_tags(_u8(c), c.size), "strip_tags")
    return c


# -------------------------------------------------------------------- FNV

def fnv1a64(x, h: int = FNV_BASIS) -> int:
    x = _arr(x)
    if x.size == 0:
        return h
    return int(lib().oracle_fnv1a64(_u8(x), x.size, h))


def fnv_chunked(x) -> int:
    x = _arr(x)
    if x.size == 0:
        x1 = np.zeros(1, dtype=np.uint8)
        return int(lib().oracle_fnv_chunked(_u8(x1), 0))
    return int(lib().oracle_fnv_chunked(_u8(x), x.size))


# ------------------------------------------------------- ratio and stats

def est_bytes(c) -> float:
    c = _arr(c)
    v = ctypes.c_double(0)
    _check(lib().oracle_est_bytes(_u8(c), c.size, ctypes.byref(v)), "est_bytes")
    return float(v.value)


@dataclass
class Stats:
    matches: int
    match_bytes: int
    literal_bytes: int
    lt16: int
    lt32: int
    per_class: tuple
    tokens: int
    blocks: int
    total_len: int

    @property
    def mean_match_len(self) -> float:
        return self.match_bytes / self.matches if self.matches else 0.0

    @property
    def coverage(self) -> float:
        return self.match_bytes / self.total_len if self.total_len else 0.0


def stats(c) -> Stats:
    c = _arr(c)
    o = np.zeros(12, dtype=np.uint64)
    _check(lib().oracle_stats(_u8(c), c.size, o.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "stats")
    o = [int(v) for v in o]
    return Stats(o[0], o[1], o[2], o[3], o[4], tuple(o[5:9]), o[9], o[10], o[11])


# ----------------------------------------------------- container reading

@dataclass
class Header:
    flags: int
    total_len: int
    block_size: int
    n_blocks: int
    n_tokens: int
    n_literals: int
    n_waves: int
    mm: tuple


def header(c) -> Header:
    b = bytes(_arr(c)[:64])
    if b[:4] != b"ACLZ":
        raise OracleError(E_CORRUPT, "header")
    ver, flags, total, bs, nb, nt, nl, nw = struct.unpack_from("<HHQIIQQI", b, 4)
    return Header(flags, total, bs, nb, nt, nl, nw, tuple(b[44:48]))


def tokens(c):
    """(lit_len, match_len, src, wave) arrays and per-block token counts."""
    c = _arr(c)
    h = header(c)
    d0 = 64
    t0 = d0 + 32 * h.n_blocks
    dirr = c[d0:t0].view(np.uint8).reshape(h.n_blocks, 32) if h.n_blocks else np.zeros((0, 32), np.uint8)
    blk_ntok = dirr[:, 16:20].copy().view(np.uint32).reshape(-1) if h.n_blocks else np.zeros(0, np.uint32)
    tok = c[t0:t0 + 16 * h.n_tokens].copy().view(np.uint32).reshape(h.n_tokens, 4)
    ll = tok[:, 0].copy()
    ml = tok[:, 1].copy()
    sw = tok[:, 2:4].copy().view(np.uint64).reshape(-1)
    src = sw & np.uint64((1 << 40) - 1)
    wave = (sw >> np.uint64(40)).astype(np.uint32)
    lits = c[t0 + 16 * h.n_tokens:].copy()
    return blk_ntok, ll, ml, src, wave, lits


# --------------------------------------------- pure-Python brute force

def dist_class(d: int) -> int:
    if d < DIST_BOUNDS[0]:
        return 0
    if d < DIST_BOUNDS[1]:
        return 1
    if d < DIST_BOUNDS[2]:
        return 2
    return 3


def brute_greedy(x: bytes, block_size: int, mm=PRESET_BASE):
    """Greedy parse by exhaustive search over all earlier positions (no
    chains, no depth or window limit): the longest valid candidate, ties to
    the nearest.  Returns per-block token lists [(lit, mlen, src)]."""
    n = len(x)
    out = []
    for b0 in range(0, n, block_size):
        bend = min(b0 + block_size, n)
        toks, p, ls = [], b0, b0
        while p < bend:
            best, bsrc = 0, 0
            if p + 4 <= n:
                for s in range(p - 1, -1, -1):
                    if x[s:s + 4] != x[p:p + 4]:
                        continue
                    d = p - s
                    lim = min(d, bend - p)
                    ln = 0
                    while ln < lim and x[s + ln] == x[p + ln]:
                        ln += 1
                    if ln >= mm[dist_class(d)] and ln > best:
                        best, bsrc = ln, s
            if best:
                toks.append((p - ls, best, bsrc))
                p += best
                ls = p
            else:
                p += 1
        if ls < bend or not toks:
            toks.append((bend - ls, 0, 0))
        out.append(toks)
    return out


def dp_min_tokens(x: bytes, block_size: int, mm=PRESET_BASE):
    """Exact minimum-token parse of each block by dynamic programming over
    every valid match (any earlier source, any length within the rules).
    Returns per-block token lists of one optimal parse."""
    n = len(x)
    out = []
    for b0 in range(0, n, block_size):
        bend = min(b0 + block_size, n)
        L = bend - b0
        INF = 1 << 30
        # best[i] = (tokens, parse) for the block suffix starting at b0 + i
        # with no pending literals; a token = literal run + match, or a
        # final literal run.
        best = [None] * (L + 1)
        best[L] = (0, [])
        for i in range(L - 1, -1, -1):
            cand = (1, [(L - i, 0, 0)])  # all remaining bytes literal
            for lit in range(0, L - i):
                p = b0 + i + lit
                for s in range(0, p):
                    d = p - s
                    lim = min(d, bend - p)
                    ln = 0
                    while ln < lim and x[s + ln] == x[p + ln]:
                        ln += 1
                    for m in range(mm[dist_class(d)], ln + 1):
                        j = i + lit + m
                        if best[j] is None:
                            continue
                        tot = 1 + best[j][0]
                        if tot < cand[0]:
                            cand = (tot, [(lit, m, s)] + best[j][1])
            best[i] = cand
        out.append(best[0][1] if L else [])
    return out


def pack_token_lists(x_len: int, block_size: int, blocks, literals_of) -> np.ndarray:
    """Container from per-block token lists; literals taken from x."""
    blk, ll, ml, sr = [], [], [], []
    for toks in blocks:
        blk.append(len(toks))
        for (a, b, c) in toks:
            ll.append(a)
            ml.append(b)
            sr.append(c)
    return pack(x_len, block_size, blk, ll, ml, sr, literals_of)


def literal_bytes(x: bytes, block_size: int, blocks) -> bytes:
    out = bytearray()
    pos = 0
    for toks in blocks:
        for (a, b, c) in toks:
            out += x[pos:pos + a]
            pos += a + b
    return bytes(out)


def simulate_waves(c, order: str = "forward", seed: int = 0) -> np.ndarray:
    """Wave-by-wave decode that runs the blocks of each wave in the given
    order (forward, reverse or shuffled) and raises if any read sees a byte
    that the wave rule does not guarantee final: a cross-block source byte
    must have been written in an earlier wave, a same-block one earlier in
    the same block.  Returns the decoded bytes."""
    h = header(c)
    blk, ll, ml, src, wave, lits = tokens(c)
    n = h.total_len
    out = np.zeros(n, dtype=np.uint8)
    written = np.full(n, -1, dtype=np.int64)
    tok_off = np.concatenate([[0], np.cumsum(blk.astype(np.int64))])
    # per-token dst and literal offset by a plain running sum
    dst = np.zeros(h.n_tokens, dtype=np.int64)
    loff = np.zeros(h.n_tokens, dtype=np.int64)
    pos, lp = 0, 0
    for i in range(h.n_tokens):
        dst[i], loff[i] = pos, lp
        pos += int(ll[i]) + int(ml[i])
        lp += int(ll[i])
    rng = np.random.default_rng(seed)
    W = int(wave.max()) + 1 if h.n_tokens else 0
    for w in range(W):
        order_b = list(range(h.n_blocks))
        if order == "reverse":
            order_b.reverse()
        elif order == "shuffle":
            rng.shuffle(order_b)
        for b in order_b:
            bstart = b * h.block_size
            bend = bstart + h.block_size
            for i in range(int(tok_off[b]), int(tok_off[b + 1])):
                d = int(dst[i])
                if w == 0:
                    a = int(ll[i])
                    out[d:d + a] = lits[loff[i]:loff[i] + a]
                    written[d:d + a] = 0
                if ml[i] and int(wave[i]) == w:
                    s, m = int(src[i]), int(ml[i])
                    d += int(ll[i])
                    for k in range(m):
                        p = s + k
                        same = bstart <= p < bend
                        ok = written[p] >= 0 and (written[p] <= w if same else written[p] < w)
                        if not ok:
                            raise OracleError(E_CORRUPT, f"simulate_waves: token {i} reads byte {p} early")
                        out[d + k] = out[p]
                        written[d + k] = w
    if n and (written < 0).any():
        raise OracleError(E_CORRUPT, "simulate_waves: bytes never written")
    return out


# ------------------------------------------------------ tile entropy layer
#
# ``ans.c``: order-0 interleaved rANS over 64 KiB tiles (32 states, M = 2^12,
# 16-bit renormalisation), our reading of the paper's tile-ANS entropy layer
# (Sec. II), and the "ACLE" container that codes a v1 container's 16 token
# byte planes and literal bytes by tiles.  Pinned in ``tests/test_ans_oracle.py``
# by round trips, the frequency rules, exact word counts in closed form, the
# Shannon lower bound and an upper bound on the code length.

ANS_M = 1 << 12
ANS_L = 1 << 16
ANS_LANES = 32
ANS_TILE = 1 << 16
ANS_TILE_HEADER = 512 + 4 * ANS_LANES + 4


def ans_quantize(counts) -> np.ndarray:
    """Tile frequencies (sum ANS_M) from 256 byte counts."""
    cnt = np.ascontiguousarray(counts, dtype=np.uint64)
    if cnt.size != 256:
        raise OracleError(E_INVAL, "ans_quantize")
    f = np.zeros(256, dtype=np.uint16)
    _check(lib().oracle_ans_quantize(cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), int(cnt.sum()),
                                     f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))), "ans_quantize")
    return f


def ans_encode_tile(x) -> np.ndarray:
    """One tile (at most 64 KiB) to its payload: freq[256], state[32], n_words, words."""
    x = _arr(x)
    cap = int(lib().oracle_ans_tile_bound(x.size))
    out = np.zeros(cap, dtype=np.uint8)
    size = ctypes.c_uint64(0)
    _check(lib().oracle_ans_encode_tile(_u8(x), x.size, _u8(out), cap, ctypes.byref(size)), "ans_encode_tile")
    return out[:size.value].copy()


def ans_decode_tile(payload, n: int) -> np.ndarray:
    p = _arr(payload)
    out = np.zeros(max(1, n), dtype=np.uint8)
    _check(lib().oracle_ans_decode_tile(_u8(p), p.size, _u8(out), n), "ans_decode_tile")
    return out[:n]


@dataclass
class AnsTile:
    freq: np.ndarray    # uint16[256]
    states: np.ndarray  # uint32[32], the decoder's starting states
    words: np.ndarray   # uint16, in decode order


def ans_tile_fields(payload) -> AnsTile:
    p = _arr(payload)
    freq = p[:512].view(np.uint16).copy()
    states = p[512:512 + 4 * ANS_LANES].view(np.uint32).copy()
    nw = int(p[512 + 4 * ANS_LANES:ANS_TILE_HEADER].view(np.uint32)[0])
    words = p[ANS_TILE_HEADER:ANS_TILE_HEADER + 2 * nw].view(np.uint16).copy()
    return AnsTile(freq, states, words)


def acle_encode(c) -> np.ndarray:
    """The entropy-coded (ACLE) form of a v1 container."""
    c = _arr(c)
    bound = ctypes.c_uint64(0)
    _check(lib().oracle_acle_bound(_u8(c), c.size, ctypes.byref(bound)), "acle_bound")
    out = np.zeros(bound.value, dtype=np.uint8)
    size = ctypes.c_uint64(0)
    _check(lib().oracle_acle_encode(_u8(c), c.size, _u8(out), out.size, ctypes.byref(size)), "acle_encode")
    return out[:size.value].copy()


def acle_decode(e) -> np.ndarray:
    """The v1 container an ACLE holds."""
    e = _arr(e)
    n = int(lib().oracle_acle_decoded_size(_u8(e), e.size))
    if n == 0:
        raise OracleError(E_CORRUPT, "acle_decode")
    out = np.zeros(n, dtype=np.uint8)
    _check(lib().oracle_acle_decode(_u8(e), e.size, _u8(out), n), "acle_decode")
    return out


@dataclass
class AcleLayout:
    size: int
    prefix: int
    n_tokens: int
    n_literals: int
    n_tiles: int
    payload_offset: int
    streams: list       # (length, first tile) per stream: 16 token planes, literals
    tiles: np.ndarray   # per tile: (payload offset, payload bytes, symbols)


def acle_layout(e) -> AcleLayout:
    e = _arr(e)
    magic, ver, size, prefix, ns, tile, nt, nl, ntl, po = struct.unpack_from("<4sIQQIIQQQQ", bytes(e[:64]))
    if magic != b"ACLE" or ver != 1:
        raise OracleError(E_CORRUPT, "acle_layout")
    st = 64 + (prefix + 15) // 16 * 16
    streams = [struct.unpack_from("<QQ", bytes(e[st + 16 * k:st + 16 * k + 16])) for k in range(ns)]
    tt = st + 16 * ns
    raw = e[tt:tt + 16 * ntl].view(np.uint32).reshape(-1, 4)
    tiles = np.stack([raw[:, 0].astype(np.uint64) | (raw[:, 1].astype(np.uint64) << 32),
                      raw[:, 2].astype(np.uint64), raw[:, 3].astype(np.uint64)], axis=1) if ntl else \
        np.zeros((0, 3), dtype=np.uint64)
    return AcleLayout(size, prefix, nt, nl, ntl, po, streams, tiles)
