"""GPU parity of read-level FASTQ seeks: reads picked by id decode, in one
batched range launch, to exactly their bytes in the input (and the oracle's
decode of the container), including the first read, the truncated last
one and reads that cross LZ block boundaries."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, synth
from paper_2607_18541_gb300.fastq_index import ReadIndex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("preset", [aclz.ACLZ_PRESET_BASE, aclz.ACLZ_PRESET_TUNED])
def test_read_seeks_equal_the_input(preset):
    x = synth.fastq(3 << 20, seed=53)
    p = aclz.aclz_encode_params_default(preset)
    p.block_size = 1 << 14
    c = aclz.aclz_encode(x, p)
    assert np.array_equal(oracle.decode(c), x)
    idx = ReadIndex.build(x)
    rng = np.random.default_rng(54)
    ids = [0, idx.n_reads - 1] + list(rng.choice(idx.n_reads, 60, replace=False))
    crossing = [i for i in range(idx.n_reads) if idx.block(i, 1 << 14) != (idx.span(i)[1] - 1) >> 14][:5]
    assert crossing
    ids += crossing
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s, flags=aclz.ACLZ_UPLOAD_FLATTEN)
    try:
        parts = idx.seek(h, ids, stream=s)
        torch.cuda.synchronize()
        for i, part in zip(ids, parts):
            lo, hi = idx.span(i)
            assert np.array_equal(part.cpu().numpy(), x[lo:hi]), i
    finally:
        aclz.aclz_free(h)
