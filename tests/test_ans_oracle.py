"""Pins of the oracle's tile entropy layer (oracle/ans.c): order-0 rANS with
32 interleaved states over 64 KiB tiles (our reading of the paper's tile-ANS
stage, Sec. II), and the ACLE container that codes a v1 container's token
byte planes and literal bytes by tiles.

What pins it, besides round trips:
  - the frequency rule worked by hand on small count vectors;
  - closed forms: a one-symbol tile emits no words and leaves every state at
    L = 2^16; a tile holding all 256 byte values equally often (f = 16 each,
    8 bits per symbol) emits exactly floor(k/2) words on a state that codes
    k symbols;
  - two-sided bounds on the code length from the rANS step itself: with
    I = sum_i log2(M / f(s_i)) the ideal information of the tile under its
    own table, the bits held (16 per word plus log2 of every final state)
    lie within I + 512 +- 0.094 (n + words), 512 being the 32 starting states
    of 16 bits;
  - the Shannon bound: I >= n H0 of the tile, so no tile codes below its
    order-0 entropy by more than those constants.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import synth

M, L, W = oracle.ANS_M, oracle.ANS_L, oracle.ANS_LANES


def _tile_bits(payload):
    t = oracle.ans_tile_fields(payload)
    return 16 * t.words.size + sum(math.log2(int(s)) for s in t.states), t


def _info(x, freq):
    f = freq.astype(np.float64)
    return float(np.sum(np.log2(M / f[x]))) if x.size else 0.0


def _h0_bits(x):
    if x.size == 0:
        return 0.0
    p = np.bincount(x, minlength=256).astype(np.float64)
    p = p[p > 0] / x.size
    return float(-(p * np.log2(p)).sum() * x.size)


# ------------------------------------------------------------ frequencies

def test_quantize_rule_by_hand():
    c = np.zeros(256, np.uint64)
    c[[0, 1, 2]] = 1                       # 4096 / 3 = 1365 each, 1 left over to the first
    f = oracle.ans_quantize(c)
    assert (f[0], f[1], f[2]) == (1366, 1365, 1365) and f.sum() == M
    c = np.zeros(256, np.uint64)
    c[7] = 10                              # one distinct symbol takes all of M
    assert oracle.ans_quantize(c)[7] == M
    c = np.full(256, 3, np.uint64)         # all equal: 16 each
    assert np.all(oracle.ans_quantize(c) == 16)
    c = np.ones(256, np.uint64)
    c[200] = 1_000_000                     # 255 rare symbols keep 1 each
    f = oracle.ans_quantize(c)
    assert f.sum() == M and f[200] == M - 255 and np.all(np.delete(f, 200) == 1)
    c = np.zeros(256, np.uint64)
    c[[10, 20]] = [1, 3]                   # 1024 and 3072, no remainder
    f = oracle.ans_quantize(c)
    assert (f[10], f[20]) == (1024, 3072)


@pytest.mark.parametrize("seed", range(8))
def test_quantize_sums_to_m_and_keeps_every_present_symbol(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 257))
    c = np.zeros(256, np.uint64)
    c[rng.choice(256, k, replace=False)] = rng.integers(1, 10 ** int(rng.integers(1, 7)), k)
    f = oracle.ans_quantize(c)
    assert f.sum() == M
    assert np.array_equal(f > 0, c > 0)
    # close to the counts: no frequency further than the adjustment from its share
    share = c.astype(np.float64) * M / c.sum()
    assert np.all(np.abs(f - share)[c > 0] <= max(1.0, M - np.floor(share).sum() + 1) + 1)


# ------------------------------------------------------------ tiles

def _tiles():
    rng = np.random.default_rng(42)
    out = []
    for n in (0, 1, 2, 31, 32, 33, 63, 64, 65, 1000, 4097, 65535, 65536):
        out.append(("uniform", rng.integers(0, 256, n, dtype=np.uint8)))
        out.append(("geometric", np.minimum(rng.geometric(0.3, n) - 1, 255).astype(np.uint8)))
    out.append(("constant", np.full(50_000, 9, np.uint8)))
    out.append(("two", rng.choice(np.array([3, 250], np.uint8), 65536, p=[0.999, 0.001])))
    out.append(("all256", np.arange(256, dtype=np.uint8)))
    out.append(("markov", synth.markov2(65536, seed=3)))
    out.append(("fastq", synth.fastq(65536, seed=4)))
    return out


@pytest.mark.parametrize("kind,x", _tiles(), ids=lambda v: v if isinstance(v, str) else str(len(v)))
def test_tile_round_trip_and_code_length_bounds(kind, x):
    p = oracle.ans_encode_tile(x)
    assert np.array_equal(oracle.ans_decode_tile(p, x.size), x)
    bits, t = _tile_bits(p)
    assert t.freq.sum() == (M if x.size else 0)
    assert np.array_equal(t.freq > 0, np.bincount(x, minlength=256) > 0)
    assert np.all(t.states >= L)
    info = _info(x, t.freq)
    slack = 0.094 * (x.size + t.words.size) + 1e-6
    assert info + 512 - slack <= bits <= info + 512 + slack
    # the table's information is never below the tile's order-0 entropy
    assert info >= _h0_bits(x) - 1e-6


def test_one_symbol_tile_emits_nothing():
    p = oracle.ans_encode_tile(np.full(65536, 200, np.uint8))
    t = oracle.ans_tile_fields(p)
    assert t.words.size == 0 and np.all(t.states == L)
    assert p.size == oracle.ANS_TILE_HEADER


@pytest.mark.parametrize("n", [256, 256 * 7 + 0, 65536])
def test_eight_bit_tile_word_count_closed_form(n):
    rng = np.random.default_rng(n)
    x = rng.permutation(np.repeat(np.arange(256, dtype=np.uint8), n // 256))
    t = oracle.ans_tile_fields(oracle.ans_encode_tile(x))
    assert np.all(t.freq == 16)
    k = np.array([len(range(lane, n, W)) for lane in range(W)])
    assert t.words.size == int((k // 2).sum())


def test_corrupt_tiles_are_rejected():
    x = synth.markov2(65536, seed=5)
    p = oracle.ans_encode_tile(x)
    bad = p.copy()
    bad[2 * int(x[0])] ^= 1                # a frequency: the table no longer sums to M
    with pytest.raises(oracle.OracleError):
        oracle.ans_decode_tile(bad, x.size)
    with pytest.raises(oracle.OracleError):
        oracle.ans_decode_tile(p[:-2], x.size)   # a word short
    with pytest.raises(oracle.OracleError):
        oracle.ans_decode_tile(p, x.size - 1)    # words left over, states not back at L


# ------------------------------------------------------------ ACLE

def _containers():
    sw = synth.copy_sweep(1 << 20, 1 << 14, 64)
    return [
        ("markov", oracle.encode(synth.markov2(600_000, seed=6), 1 << 16)),
        ("fastq", oracle.encode(synth.fastq(400_000, seed=7), 1 << 14, oracle.PRESET_TUNED)),
        ("sweep_tagged", oracle.pack_sweep(sw, tags=True)),
        ("literal_only", oracle.encode(np.frombuffer(np.random.default_rng(1).bytes(5000), np.uint8), 1 << 12)),
        ("empty", oracle.encode(np.zeros(0, np.uint8), 1 << 12)),
    ]


@pytest.mark.parametrize("kind,c", _containers(), ids=lambda v: v if isinstance(v, str) else "")
def test_acle_round_trip_and_layout(kind, c):
    e = oracle.acle_encode(c)
    assert np.array_equal(oracle.acle_decode(e), c)
    lay = oracle.acle_layout(e)
    h = oracle.header(c)
    assert lay.size == c.size and lay.n_tokens == h.n_tokens and lay.n_literals == h.n_literals
    assert lay.prefix == 64 + 32 * h.n_blocks
    assert [s[0] for s in lay.streams] == [h.n_tokens] * 16 + [h.n_literals]
    n_t = [-(-s[0] // oracle.ANS_TILE) for s in lay.streams]
    assert lay.n_tiles == sum(n_t) and [s[1] for s in lay.streams] == list(np.cumsum([0] + n_t[:-1]))
    assert lay.payload_offset % 16 == 0 and np.all(lay.tiles[:, 0] % 16 == 0)
    # every tile decodes to its stream's bytes: token plane k, or the literals
    toks = c[lay.prefix:lay.prefix + 16 * h.n_tokens].reshape(-1, 16)
    lits = c[lay.prefix + 16 * h.n_tokens:]
    for k, (length, first) in enumerate(lay.streams):
        stream = toks[:, k] if k < 16 else lits
        for j in range(n_t[k]):
            off, size, m = (int(v) for v in lay.tiles[first + j])
            p = e[lay.payload_offset + off:lay.payload_offset + off + size]
            assert np.array_equal(oracle.ans_decode_tile(p, m), stream[j * oracle.ANS_TILE:j * oracle.ANS_TILE + m])


def test_acle_is_smaller_than_the_container_on_compressible_data():
    c = oracle.encode(synth.fastq(1 << 20, seed=8), 1 << 14, oracle.PRESET_TUNED)
    e = oracle.acle_encode(c)
    assert e.size < 0.6 * c.size


def test_corrupt_acle_is_rejected():
    c = oracle.encode(synth.markov2(200_000, seed=9), 1 << 14)
    e = oracle.acle_encode(c)
    lay = oracle.acle_layout(e)
    off, size, _ = (int(v) for v in lay.tiles[-1])
    last_end = lay.payload_offset + off + size     # the end of the last payload, before padding
    for cut in (10, 64, lay.payload_offset - 1, last_end - 1):
        with pytest.raises(oracle.OracleError):
            oracle.acle_decode(e[:cut])
    bad = e.copy()
    bad[:4] = np.frombuffer(b"ACLZ", np.uint8)
    with pytest.raises(oracle.OracleError):
        oracle.acle_decode(bad)
