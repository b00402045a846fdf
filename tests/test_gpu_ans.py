"""GPU parity of the tile entropy stage (aclz_upload_acle) against the CPU
oracle: an ACLE container written by the oracle (oracle/ans.c) is decoded
on the GPU tile by tile into the v1 layout, and the handle then decodes to
exactly the oracle's output; the upload index matches a plain upload of the
same v1 container; malformed ACLEs are rejected (integer work: bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _containers():
    return [
        ("markov", lambda: oracle.encode(synth.markov2(1 << 20, seed=21), 1 << 16)),
        ("fastq_tuned", lambda: oracle.encode(synth.fastq(2 << 20, seed=22), 1 << 14, oracle.PRESET_TUNED)),
        ("sweep64_tagged", lambda: oracle.pack_sweep(synth.copy_sweep(4 << 20, 1 << 15, 64), tags=True)),
        # more than 64K tokens: every token plane spans two tiles
        ("sweep32_untagged", lambda: oracle.pack_sweep(synth.copy_sweep(4 << 20, 1 << 15, 32), tags=False)),
        ("literal_only", lambda: oracle.encode(np.frombuffer(np.random.default_rng(2).bytes(70_000), np.uint8),
                                               1 << 12)),
    ]


def _decode(h, total):
    s = torch.cuda.current_stream()
    out = torch.empty(max(16, total + 16), dtype=torch.uint8, device="cuda")
    aclz.aclz_decode_all(h, out, stream=s)
    assert aclz.aclz_device_status(h, s) == aclz.ACLZ_OK
    return out[:total].cpu().numpy()


@pytest.mark.parametrize("kind,make", _containers(), ids=lambda v: v if isinstance(v, str) else "")
def test_acle_upload_decodes_like_the_oracle(kind, make):
    c = make()
    e = oracle.acle_encode(c)
    exp = oracle.decode(c)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload_acle(e, s)
    h0 = aclz.aclz_upload(c, s)
    try:
        a, b = aclz.aclz_handle_info(h), aclz.aclz_handle_info(h0)
        assert (a.total_len, a.n_tokens, a.n_literals, a.n_deferred, a.n_waves) == \
            (b.total_len, b.n_tokens, b.n_literals, b.n_deferred, b.n_waves)
        got = _decode(h, exp.size)
        assert np.array_equal(got, exp)
        assert aclz.aclz_fnv(torch.from_numpy(got).cuda(), got.size, stream=s) == oracle.fnv_chunked(exp)
    finally:
        aclz.aclz_free(h)
        aclz.aclz_free(h0)


def test_malformed_acle_is_rejected():
    c = oracle.encode(synth.markov2(300_000, seed=23), 1 << 14)
    e = oracle.acle_encode(c)
    lay = oracle.acle_layout(e)
    s = torch.cuda.current_stream()
    off, size, m = (int(v) for v in lay.tiles[-1])     # the literal stream's last tile
    base = lay.payload_offset + off
    bad_table = e.copy()
    freq = bad_table[base:base + 512].view(np.uint16)
    freq[int(np.argmax(freq))] -= 1                     # the table no longer sums to 2^12 (host check)
    bad_count = e.copy()
    bad_count[base + 640:base + 644] = np.frombuffer(np.uint32(1 << 20).tobytes(), np.uint8)
    bad_word = e.copy()
    nw = int(e[base + 640:base + 644].view(np.uint32)[0])
    assert nw > 8
    bad_word[base + 644 + 2 * (nw // 2)] ^= 0x5A        # a word: the states do not end at 2^16 (GPU check)
    for bad in (bad_table, bad_count, bad_word, e[:lay.payload_offset - 1]):
        with pytest.raises(aclz.AclzError) as ex:
            h = aclz.aclz_upload_acle(bad, s)
            aclz.aclz_free(h)
        assert ex.value.code == aclz.ACLZ_E_CORRUPT
    # the intact one still uploads, and the context is usable
    h = aclz.aclz_upload_acle(e, s)
    try:
        assert np.array_equal(_decode(h, oracle.header(c).total_len), oracle.decode(c))
    finally:
        aclz.aclz_free(h)
