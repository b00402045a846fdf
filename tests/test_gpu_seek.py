"""GPU range decode (seek) against the oracle: decode(x)[lo:hi] byte for
byte, single ranges and many ranges in one launch."""
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


def _containers():
    x = synth.markov2(3 << 20, seed=71)
    yield "markov", oracle.encode(x, 1 << 14, oracle.PRESET_BASE)
    sw = synth.copy_sweep((4 << 20) + 777, 1 << 13, 256, seed=72)
    yield "sweep", oracle.pack_sweep(sw, tags=False)
    yield "fastq", oracle.encode(synth.fastq(2 << 20, seed=73), 1 << 12, oracle.PRESET_TUNED)
    yield "tiny_blocks", oracle.encode(synth.markov2(100_000, seed=74), 64, (4, 4, 4, 4))


def _seek(h, lo, hi, s):
    out = torch.empty(max(16, hi - lo), dtype=torch.uint8, device="cuda")
    aclz.aclz_decode_range(h, lo, hi, out, stream=s)
    assert aclz.aclz_device_status(h, s) == 0
    return out[:hi - lo].cpu().numpy()


@pytest.mark.parametrize("name,c", list(_containers()), ids=lambda v: v if isinstance(v, str) else "")
def test_random_ranges_equal_oracle_slices(name, c):
    full = oracle.decode(c)
    n = full.size
    bs = oracle.header(c).block_size
    rng = np.random.default_rng(5)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        cases = [(0, n), (0, 1), (n - 1, n), (n // 2, n // 2), (bs - 3, bs + 5), (bs, 2 * bs)]
        for _ in range(40):
            lo = int(rng.integers(0, n))
            hi = int(min(n, lo + rng.integers(1, 200_000)))
            cases.append((lo, hi))
        for lo, hi in cases:
            if hi == lo:
                out = torch.empty(16, dtype=torch.uint8, device="cuda")
                aclz.aclz_decode_range(h, lo, hi, out, stream=s)
                continue
            got = _seek(h, lo, hi, s)
            assert np.array_equal(got, full[lo:hi]), (name, lo, hi)
    finally:
        aclz.aclz_free(h)


def test_many_ranges_in_one_launch():
    x = synth.wordtext(3 << 20, seed=75, chunk_bytes=1 << 20)
    p = aclz.aclz_encode_params_default(aclz.ACLZ_PRESET_TUNED)
    p.block_size = 1 << 16
    c = aclz.aclz_encode(x, p)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        rng = np.random.default_rng(9)
        n = x.size
        los, his, outs = [], [], []
        for _ in range(64):
            lo = int(rng.integers(0, n))
            hi = int(min(n, lo + rng.integers(0, 100_000)))
            los.append(lo)
            his.append(hi)
            outs.append(torch.empty(max(16, (hi - lo + 15) // 16 * 16), dtype=torch.uint8, device="cuda"))
        scratch = torch.empty(aclz.aclz_ranges_scratch_bytes(len(los)) + 16, dtype=torch.uint8, device="cuda")
        aclz.aclz_decode_ranges(h, los, his, outs, scratch, stream=s)
        assert aclz.aclz_device_status(h, s) == 0
        for lo, hi, o in zip(los, his, outs):
            assert np.array_equal(o[:hi - lo].cpu().numpy(), x[lo:hi])
        # alone equals in the mix
        for i in (0, 17, 63):
            if his[i] > los[i]:
                assert np.array_equal(_seek(h, los[i], his[i], s), outs[i][:his[i] - los[i]].cpu().numpy())
    finally:
        aclz.aclz_free(h)


def test_range_argument_errors():
    c = oracle.encode(synth.markov2(50_000, seed=76), 1 << 12, oracle.PRESET_BASE)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        out = torch.empty(1024, dtype=torch.uint8, device="cuda")
        for lo, hi in ((10, 5), (0, 50_001)):
            with pytest.raises(aclz.AclzError) as e:
                aclz.aclz_decode_range(h, lo, hi, out, stream=s)
            assert e.value.code == aclz.ACLZ_E_INVAL
        with pytest.raises(aclz.AclzError):
            aclz.aclz_decode_range(h, 0, 100, out.data_ptr() + 1, stream=s)
    finally:
        aclz.aclz_free(h)
