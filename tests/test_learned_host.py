"""Host-side parts of the learned per-block thresholds (no GPU): the size
estimate agrees with the oracle's, per-block costs add up to the whole
stream's order-0 cost, parse statistics agree with the oracle's token
statistics, and the candidate set holds the fallback and the base vector."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, learned, synth
from paper_2607_18541_gb300 import build as libbuild


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()
    aclz.lib()


@pytest.fixture(scope="module")
def mixed():
    # FASTQ-like records then Markov bytes: blocks that want different lengths
    return np.concatenate([synth.fastq(300_000, seed=11), synth.markov2(200_000, seed=12)])


def test_candidates_hold_the_paper_vectors():
    assert learned.CANDIDATES[learned.FALLBACK] == (12, 16, 24, 32)
    assert learned.CANDIDATES[learned.BASE] == (6, 8, 10, 12)
    assert 2 <= learned.K <= 16
    assert len(set(learned.CANDIDATES)) == learned.K
    for mm in learned.CANDIDATES:
        assert list(mm) == sorted(mm) and mm[0] >= 4


@pytest.mark.parametrize("mm", [(6, 8, 10, 12), (12, 16, 24, 32)])
def test_est_bytes_equals_oracle(mixed, mm):
    c = learned.encode(mixed, mm, block_size=1 << 14)
    assert learned.est_bytes(c) == pytest.approx(oracle.est_bytes(c), rel=1e-12)


def test_block_costs_sum_to_stream_order0_cost(mixed):
    c = learned.encode(mixed, (6, 8, 10, 12), block_size=1 << 14)
    costs = learned.block_costs(c)
    streams, nb = learned._streams(c)
    assert costs.shape == (nb,)
    want = 0.0
    for s, _ in streams:
        cnt = np.bincount(s, minlength=256).astype(np.float64)
        p = cnt[cnt > 0] / s.size
        want += float(-(cnt[cnt > 0] * np.log2(p)).sum()) / 8
    assert costs.sum() == pytest.approx(want, rel=1e-10)
    assert np.all(costs > 0)


def test_parse_features_agree_with_oracle_stats(mixed):
    bs = 1 << 14
    c = learned.encode(mixed, (6, 8, 10, 12), block_size=bs)
    f = learned.parse_features(c)
    blk, ll, ml, src, lits, _, total = learned.read_tokens(c)
    nb = blk.size
    assert f.shape == (nb, 13)
    # per block: rebuild a one-block container's statistics with the oracle
    for b in (0, nb // 2, nb - 1):
        t0 = int(blk[:b].sum())
        t1 = t0 + int(blk[b])
        pos = int(min(b * bs, total))
        nm = 0
        mbytes = 0
        lt16 = lt32 = 0
        cls = [0, 0, 0, 0]
        for i in range(t0, t1):
            pos += int(ll[i])
            if ml[i]:
                nm += 1
                mbytes += int(ml[i])
                lt16 += ml[i] < 16
                lt32 += ml[i] < 32
                cls[oracle.dist_class(pos - int(src[i]))] += 1
                pos += int(ml[i])
        blen = min(bs, total - b * bs)
        assert f[b, 0] == pytest.approx(mbytes / blen)
        if nm:
            assert f[b, 2] == pytest.approx(lt16 / nm)
            assert f[b, 3] == pytest.approx(lt32 / nm)
            assert np.allclose(f[b, 4:8], np.array(cls) / nm)
        assert f[b, 12] == pytest.approx(int(blk[b]) / (blen / 1024) / 64)
    # whole-stream totals equal the oracle's statistics
    st = oracle.stats(c)
    blen = np.minimum(bs, total - np.arange(nb) * bs)
    assert round(float((f[:, 0] * blen).sum())) == st.match_bytes


def test_read_tokens_matches_oracle_reader(mixed):
    c = learned.encode(mixed, (12, 16, 24, 32), block_size=1 << 15)
    blk, ll, ml, src, lits, bs, total = learned.read_tokens(c)
    oblk, oll, oml, osrc, _, olits = oracle.tokens(c)
    assert np.array_equal(blk, oblk) and np.array_equal(ll, oll) and np.array_equal(ml, oml)
    assert np.array_equal(src.astype(np.uint64), osrc)
    assert np.array_equal(lits, olits[:lits.size]) and lits.size == oracle.header(c).n_literals
    assert bs == 1 << 15 and total == mixed.size


def test_per_block_thresholds_encode_like_the_oracle(mixed):
    bs = 1 << 14
    nb = -(-mixed.size // bs)
    k = np.arange(nb) % learned.K
    bmm = np.array([learned.CANDIDATES[i] for i in k], dtype=np.uint8)
    got = learned.encode(mixed, block_mm=bmm, block_size=bs)
    # the host encoder leaves wave tags to the GPU upload
    want = oracle.strip_tags(oracle.encode(mixed, bs, block_mm=bmm, chain_depth=16))
    assert np.array_equal(got, want)
    assert np.array_equal(oracle.decode(got), mixed)


def test_lagrange_labels_meet_the_token_target_with_the_smallest_price():
    rng = np.random.default_rng(5)
    K, nb = learned.K, 400
    ntok = rng.integers(5, 60, (K, nb)).astype(np.float64)
    costs = rng.uniform(100, 1000, (K, nb))
    for target in (1.0, 0.95, 0.8):
        y, lam = learned.lagrange_labels(costs, ntok, target)
        want = target * ntok[learned.FALLBACK].sum()
        got = ntok[y, np.arange(nb)].sum()
        assert got <= want + 1e-9
        # each label minimises cost + lam * tokens on its block
        assert np.array_equal(y, np.argmin(costs + lam * ntok, axis=0))
        # a slightly lower price misses the target (lam is the smallest)
        if lam > 1e-6:
            y2 = np.argmin(costs + 0.99 * lam * ntok, axis=0)
            assert ntok[y2, np.arange(nb)].sum() > want - 1e-9


def test_lagrange_labels_at_zero_price_take_the_smallest_blocks():
    costs = np.array([[1.0, 5.0], [2.0, 1.0]] + [[9.0, 9.0]] * (learned.K - 2))
    ntok = np.ones_like(costs)
    y, lam = learned.lagrange_labels(costs, ntok, 1.0)
    assert lam < 1e-6 and list(y) == [0, 1]


class _FixedChoices:
    """Stands in for the trained network: returns given per-block choices."""

    def __init__(self, k):
        self.k = np.asarray(k)

    def choose(self, f, tau=0.0):
        return self.k.copy()


@pytest.mark.parametrize("kind", ["lagrange", "all_push", "all_base"])
def test_check_never_returns_a_larger_or_slower_encode(monkeypatch, mixed, kind):
    bs = 1 << 14
    nb = -(-mixed.size // bs)
    monkeypatch.setattr(learned, "features", lambda x, base, block_size=bs: np.zeros((nb, learned.N_FEATURES)))
    if kind == "lagrange":
        _, costs, ntok = (None,) + tuple(
            np.stack(v) for v in zip(*[(learned.block_costs(c), learned.read_tokens(c)[0].astype(float))
                                       for c in (learned.encode(mixed, mm, block_size=bs)
                                                 for mm in learned.CANDIDATES)]))
        k, _ = learned.lagrange_labels(costs, ntok)
    elif kind == "all_push":
        k = np.full(nb, learned.CANDIDATES.index((16, 24, 32, 48)))
    else:
        k = np.full(nb, learned.BASE)
    c, kk = learned.encode_learned(_FixedChoices(k), mixed, block_size=bs)
    fb = learned.encode(mixed, learned.CANDIDATES[learned.FALLBACK], block_size=bs)
    assert learned.est_bytes(c) <= learned.est_bytes(fb)
    assert learned.read_tokens(c)[0].sum() <= learned.read_tokens(fb)[0].sum()
    assert np.array_equal(oracle.decode(c), mixed)
    # the container's tokens are exactly those of the returned choices
    bmm = np.array([learned.CANDIDATES[j] for j in kk], dtype=np.uint8)
    want = learned.read_tokens(learned.encode(mixed, block_mm=bmm, block_size=bs))
    got = learned.read_tokens(c)
    for a, b in zip(got[:5], want[:5]):
        assert np.array_equal(a, b)


def test_time_labels_meet_the_size_budget_with_the_smallest_price():
    rng = np.random.default_rng(8)
    K, nb = learned.K, 300
    ntok = rng.integers(5, 60, (K, nb)).astype(np.float64)
    ndef = np.floor(ntok * rng.uniform(0, 1, (K, nb)))
    costs = rng.uniform(100, 1000, (K, nb))
    coef = np.array([0.002, 0.01, 1e-7])
    y, lam = learned.time_labels(costs, ntok, ndef, coef)
    t = coef[0] * ntok + coef[1] * ndef
    # no larger than the fallback's size, each label the best at its price
    assert costs[y, np.arange(nb)].sum() <= costs[learned.FALLBACK].sum() + 1e-6
    assert np.array_equal(y, np.argmin(t + lam * costs, axis=0))
    # the price is the smallest that meets the budget
    if lam > 1e-12:
        y2 = np.argmin(t + 0.98 * lam * costs, axis=0)
        assert costs[y2, np.arange(nb)].sum() > costs[learned.FALLBACK].sum() - 1e-6
    # and the labelled blocks are predicted no slower than the fallback's
    assert t[y, np.arange(nb)].sum() <= t[learned.FALLBACK].sum() + 1e-9


def test_time_model_recovers_known_coefficients():
    rng = np.random.default_rng(9)
    a, b, c = 3e-5, 2e-4, 1e-9
    samples = []
    for _ in range(40):
        tok, dfr, n = rng.uniform(1e4, 1e6), rng.uniform(0, 5e5), rng.uniform(1e7, 1e9)
        samples.append((tok, dfr, n, a * tok + b * dfr + c * n))
    got = learned.fit_time_model(samples)
    assert np.allclose(got, [a, b, c], rtol=1e-6, atol=1e-12)
