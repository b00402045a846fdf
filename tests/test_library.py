"""Host-side checks of libaclz (no GPU): the shared library loads and exports
every entry point declared in include/aclz.h, and its host encoder and
container writer give byte-identical containers to the CPU oracle."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, synth
from paper_2607_18541_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()
    aclz.lib()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(aclz_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    import ctypes
    L = ctypes.CDLL(aclz.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 15
    for name in sorted(declared):
        assert hasattr(L, name), name
    # the binding wraps every declared entry point under the same name
    assert declared <= set(aclz.exported_names())


@pytest.mark.parametrize("L,bs", [(32, 4096), (64, 1 << 15), (1024, 1 << 15), (128, 1 << 12)])
def test_pack_matches_oracle(L, bs):
    sw = synth.copy_sweep((3 << 20) + 4321, bs, L, seed=L)
    got = aclz.aclz_pack(sw.total, sw.block_size, (4, 4, 4, 4), sw.blk_ntok, sw.lit_len, sw.match_len,
                         sw.src, sw.literals)
    assert np.array_equal(got, oracle.pack_sweep(sw, tags=False))


@pytest.mark.parametrize("gen", ["markov", "fastq", "text"])
@pytest.mark.parametrize("preset", [0, 1, 2])
def test_encoder_matches_oracle(gen, preset):
    n = 1 << 20
    x = {"markov": lambda: synth.markov2(n, seed=5), "fastq": lambda: synth.fastq(n, seed=6),
         "text": lambda: synth.wordtext(n, seed=7, chunk_bytes=1 << 18)}[gen]()
    mm = (oracle.PRESET_BASE, oracle.PRESET_TUNED, oracle.PRESET_PUSH)[preset]
    for bs in (1 << 12, 1 << 16):
        p = aclz.aclz_encode_params_default(preset)
        p.block_size = bs
        got = aclz.aclz_encode(x, p, threads=3)
        assert np.array_equal(got, oracle.strip_tags(oracle.encode(x, bs, mm))), bs


def test_encoder_limits_and_block_thresholds_match_oracle():
    x = synth.markov2(600_000, seed=9)
    bs = 1 << 13
    nb = (x.size + bs - 1) // bs
    bmm = np.array([[6 + (b % 5), 8 + (b % 3), 10 + b % 7, 12 + b % 11] for b in range(nb)],
                   dtype=np.uint8)
    for depth, window in ((1, 1 << 40), (8, 3000), (64, 70000), (200, 1 << 40)):
        p = aclz.aclz_encode_params_default(0)
        p.block_size, p.chain_depth, p.window = bs, depth, window
        got = aclz.aclz_encode(x, p, block_min_match=bmm, threads=4)
        exp = oracle.strip_tags(oracle.encode(x, bs, oracle.PRESET_BASE, block_mm=bmm, chain_depth=depth,
                                              window=window))
        assert np.array_equal(got, exp), (depth, window)
        assert oracle.check_thresholds(exp) == 0


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 63, 64, 65, 1000])
def test_encoder_edge_sizes_match_oracle(n):
    x = synth.markov2(max(n, 1), seed=2)[:n]
    p = aclz.aclz_encode_params_default(0)
    p.block_size = 64
    got = aclz.aclz_encode(x, p)
    assert np.array_equal(got, oracle.strip_tags(oracle.encode(x, 64, oracle.PRESET_BASE)))


def test_container_info_and_argument_errors():
    x = synth.fastq(100_000, seed=3)
    p = aclz.aclz_encode_params_default(1)
    p.block_size = 1 << 14
    c = aclz.aclz_encode(x, p)
    info = aclz.aclz_container_info(c)
    h = oracle.header(c)
    assert (info.total_len, info.n_blocks, info.n_tokens, info.block_size) == \
        (h.total_len, h.n_blocks, h.n_tokens, h.block_size)
    assert tuple(info.min_match) == oracle.PRESET_TUNED
    bad = aclz.aclz_encode_params_default(0)
    bad.block_size = 3000  # not a power of two
    with pytest.raises(aclz.AclzError) as e:
        aclz.aclz_encode(x, bad)
    assert e.value.code == aclz.ACLZ_E_INVAL
    bad = aclz.aclz_encode_params_default(0)
    bad.min_match[0] = 3
    with pytest.raises(aclz.AclzError):
        aclz.aclz_encode(x, bad)
    with pytest.raises(aclz.AclzError) as e:
        aclz.aclz_container_info(c[:40])
    assert e.value.code == aclz.ACLZ_E_CORRUPT
    with pytest.raises(aclz.AclzError):
        aclz.aclz_encode_params_default(7)


def test_batch_merge_matches_oracle_decode():
    xs = [synth.markov2(n, seed=i)[:n] if n else np.zeros(0, np.uint8)
          for i, n in enumerate((1000, 70000, 0, 65536, 123457))]
    cs = [oracle.encode(x, 4096, oracle.PRESET_BASE) for x in xs]
    merged, offs = aclz.aclz_batch_merge(cs)
    assert oracle.validate(merged) == 0
    full = oracle.decode(merged)
    for x, o in zip(xs, offs):
        assert int(o) % 4096 == 0
        assert np.array_equal(full[int(o):int(o) + x.size], x)
    stripped, _ = aclz.aclz_batch_merge([oracle.strip_tags(c) for c in cs])
    assert oracle.header(stripped).flags == 0
    assert np.array_equal(oracle.decode(stripped), full)


def test_lanes_law_follows_table_one():
    # Table I: normalised throughput 0.31 at 32K lanes, ~0.52 at 65K,
    # ~0.8 at 131K, 1.0 at >= 1M lanes
    from paper_2607_18541_gb300 import autotune
    assert abs(autotune.lanes_law(32_768) - 0.31) < 1e-9
    assert abs(autotune.lanes_law(65_536) - 0.525) < 1e-9
    assert abs(autotune.lanes_law(131_072) - 0.81) < 1e-9
    assert autotune.lanes_law(1 << 20) == 1.0 and autotune.lanes_law(1 << 24) == 1.0
    xs = [1 << k for k in range(10, 24)]
    vals = [autotune.lanes_law(x) for x in xs]
    assert all(b >= a for a, b in zip(vals, vals[1:]))
