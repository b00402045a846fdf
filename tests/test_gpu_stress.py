"""Randomised parity sweep through the C ABI: random generators, sizes,
block sizes and threshold vectors; every decode mode and group width, the
flattened and the reshaped schedules, seeks and FNV, each against the CPU
oracle (integer work: bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = ((aclz.ACLZ_MODE_WAVES, 0), (aclz.ACLZ_MODE_PERSISTENT, aclz.ACLZ_FLAG_STAGED),
         (aclz.ACLZ_MODE_PERSISTENT, aclz.ACLZ_FLAG_REGISTERS), (aclz.ACLZ_MODE_AUTO, 0))
VECTORS = ((4, 4, 4, 4), (6, 8, 10, 12), (12, 16, 24, 32), (16, 24, 32, 48), (5, 9, 13, 20))


def _case(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300_000))
    kind = int(rng.integers(0, 4))
    if kind == 0:
        x = synth.markov2(n, seed=seed)
    elif kind == 1:
        x = synth.fastq(n, seed=seed)
    elif kind == 2:
        x = synth.wordtext(n, seed=seed, chunk_bytes=1 << 20)
    else:  # runs and repeats of a small alphabet
        x = np.repeat(rng.integers(0, 4, n // 8 + 1, dtype=np.uint8), 8)[:n].copy()
    bs = 1 << int(rng.integers(6, 17))
    mm = VECTORS[int(rng.integers(0, len(VECTORS)))]
    return x, bs, mm, rng


@pytest.mark.parametrize("seed", range(24))
def test_random_streams_every_schedule(seed):
    x, bs, mm, rng = _case(seed)
    c = oracle.strip_tags(oracle.encode(x, bs, mm, chain_depth=8))
    assert np.array_equal(oracle.decode(c), x)
    fe = oracle.fnv_chunked(x)
    s = torch.cuda.current_stream()
    out = torch.empty(x.size + 16, dtype=torch.uint8, device="cuda")
    for step in ("plain", "reshape", "flatten"):
        h = aclz.aclz_upload(c, s)
        try:
            if step == "reshape":
                aclz.aclz_reshape(h, 1 + seed % 2, s)
            elif step == "flatten":
                aclz.aclz_flatten(h, s)
            for G in (8, 16, 32):
                for mode, flags in MODES:
                    out.zero_()
                    aclz.aclz_decode_all(h, out, G=G, mode=mode, flags=flags, ctas_per_sm=int(rng.integers(0, 3)),
                                         stream=s)
                    assert aclz.aclz_device_status(h, s) == 0
                    assert np.array_equal(out[:x.size].cpu().numpy(), x), (step, G, mode, flags)
            assert aclz.aclz_fnv(out, x.size, stream=s) == fe
            lo = int(rng.integers(0, x.size))
            hi = int(rng.integers(lo, x.size + 1))
            part = torch.empty(max(16, hi - lo + 16), dtype=torch.uint8, device="cuda")
            aclz.aclz_decode_range(h, lo, hi, part, stream=s)
            assert np.array_equal(part[:hi - lo].cpu().numpy(), x[lo:hi]), step
        finally:
            aclz.aclz_free(h)
