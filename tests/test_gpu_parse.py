"""GPU greedy parse (aclz_encode_gpu) against the CPU oracle's encoder:
the container must be byte for byte the one the oracle writes (without its
wave tags, as the library's host encoder writes it), on the generated
workloads at every threshold preset, with per-block thresholds, a bounded
window, chain depths below, at and above one warp of candidates, tiny and
ragged inputs, and 64-byte blocks."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    aclz.lib()


def _params(bs, mm, depth=64, window=None):
    p = aclz.aclz_encode_params_default(0)
    p.block_size = bs
    for i in range(4):
        p.min_match[i] = mm[i]
    p.chain_depth = depth
    if window is not None:
        p.window = window
    return p


def _want(x, bs, mm, depth=64, window=oracle.UNLIMITED_WINDOW, block_mm=None):
    return oracle.strip_tags(oracle.encode(x, bs, mm, block_mm=block_mm, chain_depth=depth, window=window))


PRESETS = {"base": oracle.PRESET_BASE, "tuned": oracle.PRESET_TUNED, "pushed": oracle.PRESET_PUSH}


@pytest.mark.parametrize("preset", list(PRESETS))
@pytest.mark.parametrize("name", ["markov", "fastq", "wordtext"])
def test_gpu_parse_equals_the_oracle_encoder(name, preset):
    make = {"markov": lambda: synth.markov2(3 << 20, seed=91),
            "fastq": lambda: synth.fastq(3 << 20, seed=92),
            "wordtext": lambda: synth.wordtext(2 << 20, seed=93, chunk_bytes=1 << 20)}[name]
    x = make()
    mm = PRESETS[preset]
    bs = 1 << 14
    got = aclz.aclz_encode_gpu(x, _params(bs, mm))
    assert np.array_equal(got, _want(x, bs, mm))
    # and the same bytes as the library's host encoder
    assert np.array_equal(got, aclz.aclz_encode(x, _params(bs, mm)))


@pytest.mark.parametrize("depth", [1, 31, 32, 33, 100])
def test_chain_depths_around_one_warp(depth):
    x = synth.markov2(1 << 20, seed=94)
    got = aclz.aclz_encode_gpu(x, _params(1 << 12, oracle.PRESET_BASE, depth=depth))
    assert np.array_equal(got, _want(x, 1 << 12, oracle.PRESET_BASE, depth=depth))


def test_window_and_per_block_thresholds():
    x = synth.wordtext(1 << 20, seed=95, chunk_bytes=1 << 19)
    bs = 1 << 13
    nb = -(-x.size // bs)
    rng = np.random.default_rng(96)
    cands = np.array([oracle.PRESET_BASE, oracle.PRESET_TUNED, oracle.PRESET_PUSH, (4, 4, 4, 4)], dtype=np.uint8)
    bmm = cands[rng.integers(0, len(cands), nb)]
    got = aclz.aclz_encode_gpu(x, _params(bs, oracle.PRESET_TUNED, window=20000), block_min_match=bmm)
    want = _want(x, bs, oracle.PRESET_TUNED, window=20000, block_mm=bmm)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 63, 64, 65, 1000, 65537])
def test_edge_sizes_and_64_byte_blocks(n):
    rng = np.random.default_rng(n + 97)
    # runs of a few symbols: many matches, including ones that end at block ends
    x = np.repeat(rng.integers(0, 3, n, dtype=np.uint8), rng.integers(1, 9, n))[:n].copy()
    for bs in (64, 1 << 12):
        got = aclz.aclz_encode_gpu(x, _params(bs, (4, 4, 4, 4), depth=8))
        assert np.array_equal(got, _want(x, bs, (4, 4, 4, 4), depth=8))
        assert np.array_equal(oracle.decode(got), x)


def test_gpu_parse_rejects_bad_arguments():
    x = np.zeros(100, dtype=np.uint8)
    with pytest.raises(aclz.AclzError):
        aclz.aclz_encode_gpu(x, _params(1000, oracle.PRESET_BASE))  # block size not a power of two
    with pytest.raises(aclz.AclzError):
        aclz.aclz_encode_gpu(x, _params(1 << 12, (3, 8, 10, 12)))  # minimum below 4
