"""Batched decode (one persistent launch over many merged streams, graph
captured) against the original stream bytes and the single-stream decode."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, batched, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    aclz.lib()


@pytest.mark.parametrize("mode", ["auto", "persistent", "waves"])
def test_batched_equals_streams_and_single_stream_decode(mode):
    streams = batched.make_streams(48, 16 << 10, 1 << 20, seed=123)
    p = aclz.aclz_encode_params_default(aclz.ACLZ_PRESET_TUNED)
    p.block_size = 1 << 13
    cs = batched.encode_streams(streams, p)
    cfg = {"auto": {}, "persistent": dict(mode=aclz.ACLZ_MODE_PERSISTENT, flags=aclz.ACLZ_FLAG_STAGED),
           "waves": dict(mode=aclz.ACLZ_MODE_WAVES)}[mode]
    s = torch.cuda.current_stream()
    dec = batched.BatchDecoder(cs, stream=s)
    try:
        dec.decode(**cfg)
        assert aclz.aclz_device_status(dec.h, s) == 0
        for i, x in enumerate(streams):
            assert np.array_equal(dec.stream_output(i).cpu().numpy(), x), i
        # graph replay gives the same bytes
        dec.out.zero_()
        dec.capture(**cfg)
        dec.replay()
        dec.replay()
        assert aclz.aclz_device_status(dec.h, s) == 0
        for i, x in enumerate(streams):
            assert np.array_equal(dec.stream_output(i).cpu().numpy(), x), i
        # each stream alone (single-stream decode) equals its slice of the batch
        ms, outs = batched.time_one_by_one(cs[:8], stream=s, reps=1, **cfg)
        for i in range(8):
            n = streams[i].size
            assert torch.equal(outs[i][:n], dec.stream_output(i))
    finally:
        dec.close()


def test_merged_oracle_tags_are_kept_and_decoded():
    xs = [synth.fastq(n, seed=i) for i, n in enumerate((5000, 80000, 33333))]
    cs = [oracle.encode(x, 4096, oracle.PRESET_BASE) for x in xs]
    merged, offs = aclz.aclz_batch_merge(cs)
    assert oracle.header(merged).flags == 1 and oracle.validate(merged) == 0
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(merged, s)
    try:
        n = aclz.aclz_handle_info(h).total_len
        out = torch.empty((n + 15) // 16 * 16, dtype=torch.uint8, device="cuda")
        aclz.aclz_decode_all(h, out, stream=s)
        got = out.cpu().numpy()
        for x, o in zip(xs, offs):
            assert np.array_equal(got[int(o):int(o) + x.size], x)
    finally:
        aclz.aclz_free(h)


def test_autotune_on_a_merged_batch_and_decode_with_its_choice():
    from paper_2607_18541_gb300 import autotune
    streams = batched.make_streams(24, 16 << 10, 512 << 10, seed=77)
    total = int(sum(x.size for x in streams))

    def build(bs):
        p = aclz.aclz_encode_params_default(aclz.ACLZ_PRESET_TUNED)
        p.block_size = bs
        return aclz.aclz_batch_merge(batched.encode_streams(streams, p))[0]

    res = autotune.tune(build, total, block_sizes=(4096, 16384), Gs=(16, 32), ctas=(0, 2),
                        range_bytes=(8192,), top=2, reps=2)
    best = res["best"]
    assert best["gbs"] > 0 and len(res["trials"]) >= 2
    p = aclz.aclz_encode_params_default(aclz.ACLZ_PRESET_TUNED)
    p.block_size = best["block_size"]
    s = torch.cuda.current_stream()
    dec = batched.BatchDecoder(batched.encode_streams(streams, p), stream=s)
    try:
        aclz.aclz_set_range_bytes(dec.h, best["range_bytes"], s)
        dec.capture(G=best["G"], ctas_per_sm=best["ctas_per_sm"])
        dec.replay()
        assert aclz.aclz_device_status(dec.h, s) == 0
        for i, x in enumerate(streams):
            assert np.array_equal(dec.stream_output(i).cpu().numpy(), x), i
    finally:
        dec.close()


def test_flattened_batch_decodes_every_stream():
    streams = batched.make_streams(32, 16 << 10, 1 << 20, seed=321)
    p = aclz.aclz_encode_params_default(aclz.ACLZ_PRESET_BASE)
    p.block_size = 1 << 12
    cs = batched.encode_streams(streams, p)
    s = torch.cuda.current_stream()
    dec = batched.BatchDecoder(cs, stream=s, flatten=True)
    try:
        assert aclz.aclz_handle_info(dec.h).n_waves <= 2
        dec.capture()
        dec.replay()
        assert aclz.aclz_device_status(dec.h, s) == 0
        for i, x in enumerate(streams):
            assert np.array_equal(dec.stream_output(i).cpu().numpy(), x), i
    finally:
        dec.close()
