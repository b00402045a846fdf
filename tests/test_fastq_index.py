"""Read index for FASTQ seeks (host, no GPU): record boundaries are every
fourth newline, whatever the quality symbols; the spans tile the stream,
each holds one whole record whose header names its read, and a truncated
last record is a read of its own."""
import numpy as np

from paper_2607_18541_gb300 import synth
from paper_2607_18541_gb300.fastq_index import ReadIndex


def _records(x: bytes):
    """Plain parse, byte by byte: a record closes at every fourth newline."""
    out, start, lines = [], 0, 0
    for k, ch in enumerate(x):
        if ch == 10:
            lines += 1
            if lines % 4 == 0:
                out.append((start, k + 1))
                start = k + 1
    if start < len(x):
        out.append((start, len(x)))
    return out


def test_spans_tile_the_stream_and_name_their_reads():
    x = synth.fastq(300_000, seed=51)
    idx = ReadIndex.build(x)
    assert idx.starts[0] == 0 and idx.starts[-1] == x.size and np.all(np.diff(idx.starts) > 0)
    raw = x.tobytes()
    assert [idx.span(i) for i in range(idx.n_reads)] == _records(raw)
    for i in (0, 1, idx.n_reads // 2, idx.n_reads - 2):
        lo, hi = idx.span(i)
        rec = raw[lo:hi]
        assert rec.startswith(b"@SIM.%d\n" % (i + 1)) and rec.count(b"\n") == 4 and rec.endswith(b"\n")
    # the generator cuts the stream inside a record: the last read is that piece
    lo, hi = idx.span(idx.n_reads - 1)
    assert raw[lo:hi].startswith(b"@SIM.%d\n" % idx.n_reads) and hi == x.size


def test_quality_lines_that_start_with_at_sign():
    recs = [b"@r1\nACGT\n+\n@@@@\n", b"@r2\nTTGA\n+\n@#@#\n", b"@r3\nGG\n+\n@@"]
    x = np.frombuffer(b"".join(recs), dtype=np.uint8)
    idx = ReadIndex.build(x)
    assert idx.n_reads == 3
    got = [x[slice(*idx.span(i))].tobytes() for i in range(3)]
    assert got == recs


def test_block_of_a_read():
    x = synth.fastq(200_000, seed=52)
    idx = ReadIndex.build(x)
    for i in (0, 7, idx.n_reads - 1):
        assert idx.block(i, 1 << 14) == idx.span(i)[0] >> 14
