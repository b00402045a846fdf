"""Host side of the threshold-variant configurations (no GPU): the variant
list, and one row whose entropy-coded size is the library's ACLE of the
container (checked against the oracle's decode of it) and whose ratio is
the input size over that size."""
import numpy as np

import oracle
from paper_2607_18541_gb300 import aclz, learned, synth, thresholds
from paper_2607_18541_gb300 import build as libbuild


def test_variants_are_the_presets_then_one_band_raised():
    v = dict(thresholds.variants())
    assert v["base"] == (6, 8, 10, 12) and v["tuned"] == (12, 16, 24, 32) and v["pushed"] == (16, 24, 32, 48)
    for k in range(4):
        band = v[f"tuned+band{k}"]
        diff = [i for i in range(4) if band[i] != v["tuned"][i]]
        assert diff == [k] and band[k] == v["pushed"][k]


def test_row_reports_the_coded_size_of_the_container():
    libbuild.build()
    x = synth.fastq(300_000, seed=41)
    r = thresholds.row(x, (12, 16, 24, 32), 1 << 14, gpu=False)
    c = learned.encode(x, (12, 16, 24, 32), block_size=1 << 14)
    e = aclz.aclz_acle_encode(c)
    assert np.array_equal(oracle.acle_decode(e), c)
    assert np.array_equal(oracle.decode(c), x)
    assert r["acle_bytes"] == e.size and r["container_bytes"] == c.size
    assert abs(r["ratio"] - x.size / e.size) < 1e-4
    assert r["tokens"] == oracle.header(c).n_tokens
