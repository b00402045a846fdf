"""Host side of the plateau experiment (no GPU): the copy sweep whose match
lengths are drawn from a table is a valid container (oracle validation and
round trip), draws only lengths from the table, in the table's proportions;
a one-entry table gives exactly the fixed-length sweep; and the plateau rows
carry the stream's mean match length into the sweep."""
import numpy as np

import oracle
from paper_2607_18541_gb300 import plateau, synth


def test_length_table_sweep_is_valid_and_follows_the_table():
    table = np.array([5, 17, 17, 64, 300], np.uint32)
    sw = synth.copy_sweep_lengths(4 << 20, 1 << 14, table, seed=61)
    c = oracle.pack_sweep(sw, tags=False)
    assert oracle.validate(c) == 0
    x = oracle.decode(c)
    assert x.size == 4 << 20 and int(sw.lit_len.sum() + sw.match_len.sum()) == x.size
    m = sw.match_len[sw.match_len > 0]
    assert set(np.unique(m).tolist()) <= {5, 17, 64, 300}
    share = np.array([np.mean(m == v) for v in (5, 17, 64, 300)])
    assert np.allclose(share, [0.2, 0.4, 0.2, 0.2], atol=0.02)
    # the same seed gives the same container
    sw2 = synth.copy_sweep_lengths(4 << 20, 1 << 14, table, seed=61)
    assert np.array_equal(oracle.pack_sweep(sw2, tags=False), c)


def test_one_entry_table_is_the_fixed_length_sweep():
    for L in (32, 1024):
        a = synth.copy_sweep_lengths(2 << 20, 1 << 15, [L], seed=62)
        b = synth.copy_sweep(2 << 20, 1 << 15, L, seed=62)
        for f in ("blk_ntok", "lit_len", "match_len", "src", "literals"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), (L, f)


def test_plateau_rows_carry_the_stream_mean():
    rows = plateau.run(4, 16, 1 << 16, (12, 16, 24, 32), gpu=False)
    stream, hist, fixed = rows
    assert abs(hist["mean_match_len"] - stream["mean_match_len"]) < 0.5
    assert fixed["mean_match_len"] == round(stream["mean_match_len"])
