"""Pins of the CPU oracle against facts that do not come from the oracle:
published FNV vectors, the paper's distance bands, closed forms, brute force
and exact optimal parses on tiny inputs, adversarial wave schedules."""
import os

import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


# ------------------------------------------------------------------ FNV

def test_fnv1a64_published_vectors():
    for row in _read_golden("fnv1a64_vectors.txt"):
        lit, hx = row.rsplit(" ", 1)
        data = eval(lit)  # a bytes literal from the fixture file
        assert oracle.fnv1a64(data) == int(hx, 16), row


def test_fnv_chunked_composition():
    # one chunk: hash of (le64(fnv(x)) || le64(n)) starting from the basis
    x = synth.markov2(1000, seed=7)
    inner = oracle.fnv1a64(x)
    expect = oracle.fnv1a64(inner.to_bytes(8, "little") + (1000).to_bytes(8, "little"))
    assert oracle.fnv_chunked(x) == expect
    # three chunks, the last partial
    n = 2 * 65536 + 123
    y = synth.fastq(n, seed=9)
    h = oracle.FNV_BASIS
    for off in range(0, n, 65536):
        h = oracle.fnv1a64(oracle.fnv1a64(y[off:off + 65536]).to_bytes(8, "little"), h)
    h = oracle.fnv1a64(n.to_bytes(8, "little"), h)
    assert oracle.fnv_chunked(y) == h
    assert oracle.fnv_chunked(b"") == oracle.fnv1a64((0).to_bytes(8, "little"))


# ------------------------------------------------------- distance classes

def test_distance_bands_and_presets_match_paper():
    rows = {r.split()[0]: tuple(int(v) for v in r.split()[1:]) for r in _read_golden("distance_classes.txt")}
    assert rows["bands"] == oracle.DIST_BOUNDS
    assert rows["base"] == oracle.PRESET_BASE
    assert rows["tuned"] == oracle.PRESET_TUNED
    assert rows["push"] == oracle.PRESET_PUSH


@pytest.mark.parametrize("d,cls", [(16, 0), (127, 0), (128, 1), (16383, 1), (16384, 2),
                                   (2097151, 2), (2097152, 3), (5000000, 3)])
def test_threshold_check_uses_bands(d, cls):
    # a container whose single match sits at distance d with length T-1 then T
    T = oracle.PRESET_BASE[cls]
    for mlen, ok in ((T - 1, False), (T, True)):
        total = d + mlen
        if total > (1 << 23):
            bs = 1 << 24
        else:
            bs = 1 << 23
        lits = (np.arange(d, dtype=np.uint64) % 251).astype(np.uint8).tobytes()
        c = oracle.pack(total, bs, [1], [d], [mlen], [0], lits, mm=oracle.PRESET_BASE)
        assert oracle.validate(c) == 0
        assert (oracle.check_thresholds(c) == 0) == ok, (d, mlen)


# --------------------------------------------------------- round trips

@pytest.mark.parametrize("gen", ["markov", "fastq", "text", "zeros", "random"])
@pytest.mark.parametrize("mm", [oracle.PRESET_BASE, oracle.PRESET_TUNED, oracle.PRESET_PUSH])
def test_round_trip_and_invariants(gen, mm):
    n = 300_000
    if gen == "markov":
        x = synth.markov2(n, seed=11)
    elif gen == "fastq":
        x = synth.fastq(n, seed=12)
    elif gen == "text":
        x = synth.wordtext(n, seed=13, chunk_bytes=1 << 16)
    elif gen == "zeros":
        x = np.zeros(n, dtype=np.uint8)
    else:
        x = np.frombuffer(np.random.default_rng(5).bytes(n), dtype=np.uint8)
    bs = 16384
    c = oracle.encode(x, bs, mm)
    assert oracle.validate(c) == 0
    assert oracle.check_thresholds(c) == 0
    y = oracle.decode(c)
    assert np.array_equal(x, y)
    h = oracle.header(c)
    assert h.total_len == n and h.n_blocks == (n + bs - 1) // bs
    blk, ll, ml, src, wave, lits = oracle.tokens(c)
    # token lengths sum to each block's length; sources strictly precede targets
    tok_off = np.concatenate([[0], np.cumsum(blk.astype(np.int64))])
    dst = np.concatenate([[0], np.cumsum(ll.astype(np.int64) + ml.astype(np.int64))])[:-1] + ll
    for b in range(h.n_blocks):
        s = int((ll[tok_off[b]:tok_off[b + 1]].astype(np.int64) + ml[tok_off[b]:tok_off[b + 1]]).sum())
        assert s == min(bs, n - b * bs)
    m = ml > 0
    assert np.all(src[m].astype(np.int64) + ml[m] <= dst[m])
    assert lits.size == int(ll.sum())


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 15, 16, 17, 4095, 4096, 4097, 12289])
def test_round_trip_edge_sizes(n):
    x = synth.markov2(max(n, 1), seed=21)[:n]
    c = oracle.encode(x, 4096, oracle.PRESET_BASE)
    assert oracle.validate(c) == 0
    assert np.array_equal(oracle.decode(c), x)
    assert oracle.header(c).n_blocks == (n + 4095) // 4096


def test_window_and_depth_limits_hold():
    x = synth.markov2(200_000, seed=3)
    for depth, window in ((1, 1 << 40), (4, 5000), (64, 70000)):
        c = oracle.encode(x, 8192, oracle.PRESET_BASE, chain_depth=depth, window=window)
        assert np.array_equal(oracle.decode(c), x)
        blk, ll, ml, src, wave, lits = oracle.tokens(c)
        dst = np.concatenate([[0], np.cumsum(ll.astype(np.int64) + ml)])[:-1] + ll
        m = ml > 0
        assert np.all(dst[m] - src[m].astype(np.int64) <= window)


# ------------------------------------------------------------ brute force

def _tok_lists(c):
    blk, ll, ml, src, wave, lits = oracle.tokens(c)
    out, i = [], 0
    for n in blk:
        out.append([(int(ll[j]), int(ml[j]), int(src[j])) for j in range(i, i + int(n))])
        i += int(n)
    return out


@pytest.mark.parametrize("seed", range(40))
def test_greedy_equals_brute_force_on_tiny_inputs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 65))
    alpha = int(rng.integers(1, 4))
    x = bytes(rng.integers(0, alpha + 1, n, dtype=np.uint8))
    bs = int(rng.choice([16, 32, 48, 64]))
    mm = (4, 5, 6, 7) if seed % 2 else oracle.PRESET_BASE
    c = oracle.encode(x, bs, mm, chain_depth=oracle.UNLIMITED_DEPTH)
    assert _tok_lists(c) == oracle.brute_greedy(x, bs, mm)


@pytest.mark.parametrize("seed", range(12))
def test_optimal_parse_bounds_greedy_and_decodes(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(8, 25))
    x = bytes(rng.integers(0, 3, n, dtype=np.uint8))
    bs, mm = 16, (4, 4, 4, 4)
    greedy = oracle.brute_greedy(x, bs, mm)
    opt = oracle.dp_min_tokens(x, bs, mm)
    for g, o in zip(greedy, opt):
        assert len(g) >= len(o)
    # the optimal parse is a parse greedy never emits; it must decode to x
    lits = oracle.literal_bytes(x, bs, opt)
    c = oracle.pack_token_lists(n, bs, opt, lits)
    assert oracle.validate(c) == 0
    assert bytes(oracle.decode(c)) == x


def test_all_distinct_input_has_no_matches():
    x = np.random.default_rng(0).permutation(256).astype(np.uint8)
    c = oracle.encode(x, 256, (4, 4, 4, 4), chain_depth=oracle.UNLIMITED_DEPTH)
    st = oracle.stats(c)
    assert st.matches == 0 and st.tokens == 1 and st.literal_bytes == 256


@pytest.mark.parametrize("T0,n", [(6, 5000), (12, 3000), (16, 777)])
def test_constant_run_gives_doubling_chain(T0, n):
    # non-overlapping matches on a constant run: the first match sits at T0
    # with length T0, then each match doubles (the whole prefix is the best
    # source) until the block end caps it; a capped length is reached by every
    # distance >= the cap, and the tie goes to the nearest, src = p - len.
    x = np.full(n, 0x41, dtype=np.uint8)
    mm = (T0, T0, T0, T0)
    c = oracle.encode(x, 1 << 16, mm, chain_depth=oracle.UNLIMITED_DEPTH)
    toks = _tok_lists(c)[0]
    expect, p = [], T0
    expect.append((T0, T0, 0))
    p = 2 * T0
    while p < n:
        ln = min(p, n - p)
        if ln < T0:
            break
        expect.append((0, ln, p - ln))
        p += ln
    if p < n:
        expect.append((n - p, 0, 0))
    assert toks == expect


# ---------------------------------------------------------------- waves

@pytest.mark.parametrize("gen", ["markov", "sweep"])
def test_wave_tags_are_safe_under_any_block_order(gen):
    if gen == "markov":
        x = synth.markov2(20000, seed=31)
        c = oracle.encode(x, 1024, oracle.PRESET_BASE)
    else:
        sw = synth.copy_sweep(20000, 1024, 32, seed=32)
        c = oracle.pack_sweep(sw)
        x = oracle.decode(c)
    for order in ("forward", "reverse", "shuffle"):
        assert np.array_equal(oracle.simulate_waves(c, order, seed=1), x)


@pytest.mark.parametrize("seed", range(6))
def test_wave_tags_are_minimal(seed):
    sw = synth.copy_sweep(4096, 256, 16, seed=seed)
    c = oracle.pack_sweep(sw)
    tags, nw = oracle.min_tags(c)
    blk, ll, ml, src, wave, lits = oracle.tokens(c)
    assert np.array_equal(tags, wave)
    # lowering any single nonzero tag makes the tagging illegal
    idx = np.nonzero(tags)[0]
    rng = np.random.default_rng(seed)
    for i in rng.choice(idx, size=min(25, idx.size), replace=False):
        bad = c.copy()
        t0 = 64 + 32 * oracle.header(c).n_blocks + 16 * int(i)
        sw64 = bad[t0 + 8:t0 + 16].view(np.uint64)
        sw64[0] = np.uint64(int(sw64[0]) - (1 << 40))
        assert oracle.validate(bad) == oracle.E_CORRUPT


def test_nonminimal_tags_are_legal_and_decode_the_same():
    x = synth.markov2(50000, seed=41)
    c = oracle.encode(x, 2048, oracle.PRESET_BASE)
    h = oracle.header(c)
    extra = np.random.default_rng(0).integers(0, 3, h.n_tokens).astype(np.uint32)
    c2 = oracle.retag(c, extra)
    assert oracle.validate(c2) == 0
    assert oracle.header(c2).n_waves >= h.n_waves
    assert np.array_equal(oracle.simulate_waves(c2, "shuffle", seed=3), x)


# ------------------------------------------------------------ corruption

def test_validation_rejects_corrupt_containers():
    x = synth.markov2(20000, seed=51)
    c = oracle.encode(x, 4096, oracle.PRESET_BASE)
    h = oracle.header(c)
    t0 = 64 + 32 * h.n_blocks
    blk, ll, ml, src, wave, lits = oracle.tokens(c)
    mi = int(np.nonzero(ml)[0][3])
    cases = []
    b = c.copy(); b[0] = ord("X"); cases.append(b)                       # magic
    b = c.copy(); b[8:16] = np.frombuffer((h.total_len + 1).to_bytes(8, "little"), np.uint8); cases.append(b)
    b = c.copy(); b[t0 + 16 * mi + 4] ^= 1; cases.append(b)              # match_len
    b = c.copy()                                                          # src >= dst
    b[t0 + 16 * mi + 8:t0 + 16 * mi + 13] = np.frombuffer((h.total_len - 1).to_bytes(5, "little"), np.uint8)
    cases.append(b)
    b = c.copy(); b[64] ^= 1; cases.append(b)                             # directory tok_off
    cases.append(c[:-1].copy())                                           # truncated
    for b in cases:
        assert oracle.validate(b) < 0
    with pytest.raises(oracle.OracleError):
        oracle.decode(cases[0])


# --------------------------------------------------------- entropy estimate

def test_est_bytes_closed_forms():
    # one block, one literal-only token of 65536 identical bytes
    n = 65536
    c = oracle.pack(n, n, [1], [n], [0], [0], bytes(n))
    # header 64 + directory 32 + literal tile (H0=0) 512 + lit_len stream
    # (LEB128 of 65536 = 80 80 04: p = 2/3, 1/3) + match_len stream (one
    # zero byte) + no offsets
    lit_bits = 2 * np.log2(1.5) + np.log2(3)
    expect = 64 + 32 + 512 + (lit_bits / 8 + 512) + 512
    assert abs(oracle.est_bytes(c) - expect) < 1e-9
    # uniform literal tile: every byte value 256 times -> 8 bits per byte
    lits = bytes(np.tile(np.arange(256, dtype=np.uint8), 256))
    c = oracle.pack(n, n, [1], [n], [0], [0], lits)
    expect = 64 + 32 + (n + 512) + (lit_bits / 8 + 512) + 512
    assert abs(oracle.est_bytes(c) - expect) < 1e-9


def test_tuned_thresholds_raise_mean_match_length():
    # the lever's mechanism (Sec. IV-C): raising the minimum lengths removes
    # short matches, so the mean match length rises
    x = synth.fastq(1 << 20, seed=61)
    sb = oracle.stats(oracle.encode(x, 16384, oracle.PRESET_BASE))
    st = oracle.stats(oracle.encode(x, 16384, oracle.PRESET_TUNED))
    assert st.mean_match_len > sb.mean_match_len
    assert st.lt16 / max(1, st.matches) < sb.lt16 / max(1, sb.matches)


# -------------------------------------------------------- generator stats

def test_fastq_generator_matches_its_recipe():
    x = synth.fastq(4 << 20, seed=synth.SEED_FASTQ).tobytes()
    lines = x.split(b"\n")[:-1]
    recs = len(lines) // 4
    assert lines[0] == b"@SIM.1" and lines[4] == b"@SIM.2"
    quals = b"".join(lines[3:4 * recs:4])
    bases = b"".join(lines[1:4 * recs:4])
    assert all(len(l) == 150 for l in lines[1:4 * recs:4])
    cnt = np.bincount(np.frombuffer(quals, np.uint8), minlength=256)
    assert np.count_nonzero(cnt) == 38          # 38 quality levels (Sec. VII)
    p = cnt[cnt > 0] / cnt.sum()
    h0 = -(p * np.log2(p)).sum()
    assert abs(h0 - 3.72) < 0.15                # quality entropy 3.72 bits (Sec. VII)
    nfrac = bases.count(b"N") / len(bases)
    assert 0.0005 < nfrac < 0.002


def test_markov_repeat_rate_and_copy_sweep_recipe():
    sw = synth.copy_sweep(1 << 22, 1 << 15, 64, seed=5)
    full = sw.match_len > 0
    assert np.all(sw.match_len[full] == 64)
    assert abs(sw.lit_len[full].mean() - 4.0) < 0.1
    assert int(sw.lit_len.sum() + sw.match_len.sum()) == 1 << 22
    x = synth.markov2(1 << 20, seed=1)
    assert x.min() >= 0x30 and x.max() <= 0x6F
    # same seed, same bytes
    assert np.array_equal(x, synth.markov2(1 << 20, seed=1))


def test_stats_count_a_hand_built_parse():
    # one block holding matches at distances in every band (Sec. IV-B:
    # < 128, < 16384, < 2097152, >= 2097152) and of lengths 8 .. 100
    total = 3 << 20
    # (literal run, match length, distance)
    plan = [(2200000, 8, 100), (10, 20, 127), (3, 40, 128), (0, 8, 16383), (5, 100, 16384),
            (0, 20, 2097151), (0, 12, 2097152)]
    pos, toks = 0, []
    for ll, ml, dist in plan:
        pos += ll
        toks.append((ll, ml, pos - dist))
        pos += ml
    toks.append((total - pos, 0, 0))
    nlit = sum(t[0] for t in toks)
    lits = np.random.default_rng(8).integers(0, 256, nlit, dtype=np.uint8)
    c = oracle.pack(total, 4 << 20, [len(toks)], [t[0] for t in toks], [t[1] for t in toks],
                    [t[2] for t in toks], lits, tags=False)
    st = oracle.stats(c)
    assert st.matches == 7 and st.match_bytes == 8 + 20 + 40 + 8 + 100 + 20 + 12
    assert st.literal_bytes == nlit and st.literal_bytes + st.match_bytes == total
    assert st.lt16 == 3 and st.lt32 == 5
    assert st.per_class == (2, 2, 2, 1)
    assert st.tokens == 8 and st.blocks == 1 and st.total_len == total
