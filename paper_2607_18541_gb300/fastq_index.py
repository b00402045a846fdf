"""Read-level seek for FASTQ streams: read id -> byte range -> LZ block.

The paper's seek is read/block-level (a read id maps to the block holding
it; limits section), and absolute offsets make any byte range decodable on
its own (abstract).  A FASTQ record is four lines (header, bases, '+',
qualities), so record boundaries are every fourth newline; searching for
'@' would misfire, since '@' is also a quality symbol.  The index is built
once from the raw stream at encode time and kept next to the container;
seeks then go through the library's batched range decode.

    idx = ReadIndex.build(x)          # host, O(n)
    lo, hi = idx.span(i)              # bytes of read i (0-based record order)
    idx.block(i, block_size)          # the LZ block holding its first byte
    parts = idx.seek(h, [i, j, k])    # device buffers, one per read
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import aclz


@dataclass
class ReadIndex:
    starts: np.ndarray  # int64, n_reads + 1: record i is [starts[i], starts[i + 1])

    @staticmethod
    def build(x: np.ndarray) -> "ReadIndex":
        """Record boundaries of a FASTQ byte stream (a last, truncated record
        counts as a record)."""
        x = np.ascontiguousarray(x, dtype=np.uint8)
        nl = np.flatnonzero(x == 10)
        ends = nl[3::4] + 1  # one past the newline that closes each record
        starts = np.concatenate([[0], ends]).astype(np.int64)
        if starts[-1] != x.size:
            starts = np.concatenate([starts, [x.size]])
        return ReadIndex(starts)

    @property
    def n_reads(self) -> int:
        return int(self.starts.size - 1)

    def span(self, i: int) -> tuple[int, int]:
        if not 0 <= i < self.n_reads:
            raise IndexError(i)
        return int(self.starts[i]), int(self.starts[i + 1])

    def block(self, i: int, block_size: int) -> int:
        return self.span(i)[0] // block_size

    def seek(self, h: int, ids, stream=None):
        """Decode the given reads from an uploaded handle in one batched
        launch; returns one uint8 CUDA tensor per read (its bytes only)."""
        import torch
        ids = [int(i) for i in ids]
        spans = [self.span(i) for i in ids]
        lo = [a for a, _ in spans]
        hi = [b for _, b in spans]
        outs = [torch.empty(max(16, (b - a + 15) // 16 * 16), dtype=torch.uint8, device="cuda") for a, b in spans]
        need = aclz.aclz_ranges_scratch_bytes(len(ids))
        scratch = torch.empty(max(16, need), dtype=torch.uint8, device="cuda")
        aclz.aclz_decode_ranges(h, lo, hi, outs, scratch, stream=stream)
        return [o[:b - a] for o, (a, b) in zip(outs, spans)]
