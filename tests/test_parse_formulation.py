"""The greedy parse is block-parallel once its candidate chains are known,
and the chains are a sort: a pin of the oracle encoder by a different
formulation, and the form a GPU parse takes (R7–R8).

The oracle encoder (oracle/aclz_oracle.c) follows previous-occurrence links
built with a hash table and walks the blocks in order.  Here the candidates
of position p are read from the positions sorted by (4-byte prefix,
position): the entries just before p in that order with the same prefix,
most recent first.  Every block is then parsed on its own, in reverse block
order, and the tokens must equal the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import synth


def _sorted_chains(x: np.ndarray):
    n = x.size
    m = max(0, n - 3)
    pre = np.zeros(m, dtype=np.uint64)
    for k in range(4):
        pre |= x[k:k + m].astype(np.uint64) << np.uint64(8 * k)
    order = np.lexsort((np.arange(m), pre))  # by prefix, then by position
    rank = np.empty(m, dtype=np.int64)
    rank[order] = np.arange(m)
    return pre, order, rank


def _parse_block(x, b, bs, T, chains, depth, window):
    pre, order, rank = chains
    n = x.size
    start, end = b * bs, min((b + 1) * bs, n)
    toks, p, lit0 = [], start, start
    while p < end:
        best_len, best_src = 0, 0
        if p + 4 <= n:
            r, seen = rank[p] - 1, 0
            while r >= 0 and pre[order[r]] == pre[p] and seen < depth:
                q = int(order[r])
                if p - q > window:
                    break
                seen += 1
                lim = min(p - q, end - p)
                ln = 0
                while ln < lim and x[q + ln] == x[p + ln]:
                    ln += 1
                if ln >= T[oracle.dist_class(p - q)] and ln > best_len:
                    best_len, best_src = ln, q
                r -= 1
        if best_len:
            toks.append((p - lit0, best_len, best_src))
            p += best_len
            lit0 = p
        else:
            p += 1
    if lit0 < end or not toks:
        toks.append((end - lit0, 0, 0))
    return toks


def _cases():
    rng = np.random.default_rng(71)
    runs = np.repeat(rng.integers(0, 3, 4000, dtype=np.uint8), rng.integers(1, 12, 4000))[:30_000]
    return [
        ("markov_base", synth.markov2(40_000, seed=72), 1 << 12, oracle.PRESET_BASE, 16),
        ("fastq_tuned", synth.fastq(40_000, seed=73), 1 << 12, oracle.PRESET_TUNED, 64),
        ("runs_min4", runs.copy(), 1 << 10, (4, 4, 4, 4), 8),
        ("wordtext_push", synth.wordtext(30_000, seed=74), 1 << 11, oracle.PRESET_PUSH, 4),
    ]


@pytest.mark.parametrize("name,x,bs,mm,depth", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_sorted_chains_and_independent_blocks_reproduce_the_oracle(name, x, bs, mm, depth):
    c = oracle.encode(x, bs, mm, chain_depth=depth)
    blk, ll, ml, src, _, _ = oracle.tokens(c)
    chains = _sorted_chains(x)
    nb = -(-x.size // bs)
    got = {}
    for b in reversed(range(nb)):  # any block order: each block needs only x and the chains
        got[b] = _parse_block(x, b, bs, mm, chains, depth, window=1 << 62)
    flat = [t for b in range(nb) for t in got[b]]
    assert [len(got[b]) for b in range(nb)] == [int(v) for v in blk]
    assert [t[0] for t in flat] == [int(v) for v in ll]
    assert [t[1] for t in flat] == [int(v) for v in ml]
    assert [t[2] for t in flat if t[1]] == [int(s) for s, m in zip(src, ml) if m]
