"""Host-side checks of aclz_upload_acle (no GPU): a malformed ACLE container
or unknown flags are refused before any device work, with ACLZ_E_CORRUPT or
ACLZ_E_INVAL.  The checks cover the header, the stream and tile tables, the
payload bounds and every tile's frequency table and word count; the GPU
parity of accepted containers is in test_gpu_ans.py."""
import functools

import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, synth
from paper_2607_18541_gb300 import build as libbuild


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()
    aclz.lib()


@pytest.fixture(scope="module")
def acle():
    c = oracle.encode(synth.markov2(200_000, seed=31), 1 << 14)
    e = oracle.acle_encode(c)
    return e, oracle.acle_layout(e)


def _u32(v):
    return np.frombuffer(np.uint32(v).tobytes(), np.uint8)


def _u64(v):
    return np.frombuffer(np.uint64(v).tobytes(), np.uint8)


def _variants(e, lay):
    tt = lay.payload_offset - 16 * lay.n_tiles            # tile table
    st = tt - 16 * 17                                     # stream table
    first = lay.payload_offset + int(lay.tiles[0][0])     # first payload
    out = {}
    b = e.copy(); b[:4] = np.frombuffer(b"ACLZ", np.uint8); out["magic"] = b
    b = e.copy(); b[4:8] = _u32(2); out["version"] = b
    out["short"] = e[:40].copy()
    out["truncated_tables"] = e[:lay.payload_offset - 1].copy()
    b = e.copy(); b[8:16] = _u64(lay.size + 1); out["v1_size"] = b
    b = e.copy(); b[24:28] = _u32(16); out["n_streams"] = b
    b = e.copy(); b[28:32] = _u32(1 << 15); out["tile_size"] = b
    b = e.copy(); b[48:56] = _u64(lay.n_tiles + 1); out["n_tiles"] = b
    b = e.copy(); b[st:st + 8] = _u64(lay.n_tokens + 1); out["stream_length"] = b
    b = e.copy(); b[tt + 12:tt + 16] = _u32(7); out["tile_bytes"] = b
    b = e.copy(); b[tt:tt + 8] = _u64(8); out["unaligned_payload"] = b
    b = e.copy(); b[tt:tt + 8] = _u64(1 << 40); out["payload_out_of_range"] = b
    b = e.copy(); f = b[first:first + 512].view(np.uint16); f[int(np.argmax(f))] += 1; out["table_sum"] = b
    b = e.copy(); b[first + 640:first + 644] = _u32(1); out["word_count"] = b
    b = e.copy(); b[64 + 20:64 + 24] = _u32(3); out["v1_directory"] = b   # n_blocks of the raw v1 header
    # fields that all agree on a directory far longer than the buffer: the
    # raw header claims 2^20 blocks, and the v1 size and literal counts
    # (ACLE header and raw header) are set to match it, so only the stored
    # prefix length shows that the directory is not in the buffer
    b = e.copy()
    bs = int(b[64 + 16:64 + 20].view(np.uint32)[0])
    nb = 1 << 20
    size = 64 + 32 * nb + 16 * lay.n_tokens + (1 << 30)
    b[8:16] = _u64(size)
    b[40:48] = _u64(size - lay.prefix - 16 * lay.n_tokens)
    b[64 + 8:64 + 16] = _u64(bs * nb)
    b[64 + 20:64 + 24] = _u32(nb)
    b[64 + 32:64 + 40] = _u64(1 << 30)
    out["directory_beyond_buffer"] = b
    return out


@pytest.mark.parametrize("name", ["magic", "version", "short", "truncated_tables", "v1_size", "n_streams",
                                  "tile_size", "n_tiles", "stream_length", "tile_bytes", "unaligned_payload",
                                  "payload_out_of_range", "table_sum", "word_count", "v1_directory",
                                  "directory_beyond_buffer"])
def test_malformed_acle_is_refused_on_the_host(acle, name):
    e, lay = acle
    bad = _variants(e, lay)[name]
    with pytest.raises(aclz.AclzError) as ex:
        aclz.aclz_upload_acle(bad, None)
    assert ex.value.code == aclz.ACLZ_E_CORRUPT


def test_unknown_flags_are_refused(acle):
    e, _ = acle
    with pytest.raises(aclz.AclzError) as ex:
        aclz.aclz_upload_acle(e, None, flags=4)
    assert ex.value.code == aclz.ACLZ_E_INVAL


@functools.lru_cache(maxsize=1)
def _containers():
    return {
        "markov": oracle.encode(synth.markov2(1 << 20, seed=32), 1 << 16),
        "fastq_tuned": oracle.encode(synth.fastq(1 << 20, seed=33), 1 << 14, oracle.PRESET_TUNED),
        "sweep32_tagged": oracle.pack_sweep(synth.copy_sweep(4 << 20, 1 << 15, 32), tags=True),
        "literal_only": oracle.encode(np.frombuffer(np.random.default_rng(3).bytes(150_000), np.uint8), 1 << 12),
        "empty": oracle.encode(np.zeros(0, np.uint8), 1 << 12),
    }


@pytest.mark.parametrize("name", ["markov", "fastq_tuned", "sweep32_tagged", "literal_only", "empty"])
@pytest.mark.parametrize("threads", [0, 1, 3])
def test_library_acle_encoder_writes_the_oracles_bytes(name, threads):
    # the format fixes every byte (tables, states, word order, padding), so
    # the library's encoder and the oracle's must agree exactly
    c = _containers()[name]
    e = aclz.aclz_acle_encode(c, threads=threads)
    assert np.array_equal(e, oracle.acle_encode(c))
    assert np.array_equal(oracle.acle_decode(e), c)


def test_library_acle_encoder_refuses_bad_input():
    c = oracle.encode(synth.markov2(100_000, seed=34), 1 << 14)
    bad = c.copy()
    bad[:4] = np.frombuffer(b"ACLE", np.uint8)
    with pytest.raises(aclz.AclzError) as ex:
        aclz.aclz_acle_encode(bad)
    assert ex.value.code == aclz.ACLZ_E_CORRUPT
    bound = aclz.ctypes.c_uint64(0)
    assert aclz.lib().aclz_acle_bound(aclz._hptr(c), c.size, aclz.ctypes.byref(bound)) == 0
    out = np.zeros(64, np.uint8)
    size = aclz.ctypes.c_uint64(0)
    rc = aclz.lib().aclz_acle_encode(aclz._hptr(c), c.size, 0, aclz._hptr(out), out.size, aclz.ctypes.byref(size))
    assert rc == aclz.ACLZ_E_CAPACITY and bound.value > out.size


@pytest.mark.parametrize("name", ["markov", "empty"])
def test_valid_acle_passes_the_host_checks(name):
    # on a machine without a GPU the call then fails at device allocation,
    # never as a malformed container; with one it uploads
    e = aclz.aclz_acle_encode(_containers()[name])
    try:
        h = aclz.aclz_upload_acle(e, None)
    except aclz.AclzError as ex:
        assert ex.code not in (aclz.ACLZ_E_CORRUPT, aclz.ACLZ_E_INVAL)
    else:
        aclz.aclz_free(h)
