"""The library's host encoder (aclz_encode) writes exactly the oracle
encoder's container (greedy exact-prefix chain parse, R7–R8) at sizes where
its per-thread chain tables grow many times, for every thread count: a new
key stored in the step that grows a table must survive the rehash."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, synth
from paper_2607_18541_gb300 import build as libbuild


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


@pytest.mark.parametrize("name,preset,threads", [("markov", 0, 0), ("markov", 0, 3), ("wordtext", 1, 0),
                                                 ("fastq", 2, 5)])
def test_library_encoder_equals_the_oracle_on_large_inputs(name, preset, threads):
    make = {"markov": lambda: synth.markov2(8 << 20, seed=3), "wordtext": lambda: synth.wordtext(4 << 20, seed=4),
            "fastq": lambda: synth.fastq(4 << 20, seed=2)}[name]
    x = make()
    p = aclz.aclz_encode_params_default(preset)
    p.block_size = 1 << 14
    got = aclz.aclz_encode(x, p, threads=threads)
    mm = tuple(p.min_match[i] for i in range(4))
    want = oracle.strip_tags(oracle.encode(x, 1 << 14, mm, chain_depth=p.chain_depth))
    assert np.array_equal(got, want)
