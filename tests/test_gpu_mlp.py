"""GPU parity of the learned-threshold kernels against the float64 CPU oracle
(oracle/mlp.py): forward logits, the gradient of one batch (tiles plus the
fixed-order reduction, full and ragged batches), Adam steps, and the block
features; then training on the GPU lowers the loss, and the learned encoder
decodes bit-exactly and is never larger than the fixed 12/16/24/32 lever."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2607_18541_gb300 import aclz, learned, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _case(K, B, seed):
    rng = np.random.default_rng(seed)
    p = mlp.init(K, seed) + rng.standard_normal(mlp.n_params(K)) * 0.02
    x = rng.standard_normal((B, mlp.D))
    y = rng.integers(0, K, B)
    return p.astype(np.float32), x.astype(np.float32), y.astype(np.int32)


@pytest.mark.parametrize("K,B", [(2, 1), (12, 32), (12, 257), (16, 1000)])
def test_forward_and_gradient_match_oracle(K, B):
    p, x, y = _case(K, B, 100 + B)
    assert aclz.aclz_mlp_param_count(K) == mlp.n_params(K)
    dp, dx, dy = _dev(p), _dev(x), _dev(y, torch.int32)
    logits = torch.empty(B, K, device="cuda")
    aclz.aclz_mlp_forward(dp, K, dx, B, logits)
    z, _ = mlp.forward(p.astype(np.float64), x.astype(np.float64), K)
    assert np.allclose(logits.cpu().numpy(), z, rtol=1e-4, atol=1e-4)
    g = torch.empty(mlp.n_params(K), device="cuda")
    loss = torch.empty(1, device="cuda")
    scratch = torch.empty(aclz.aclz_mlp_scratch_bytes(K, B), dtype=torch.uint8, device="cuda")
    aclz.aclz_mlp_grad(dp, K, dx, dy, B, g, loss, scratch)
    L, gw = mlp.grads(p.astype(np.float64), x.astype(np.float64), y, K)
    assert float(loss.item()) == pytest.approx(L, rel=1e-4)
    gg = g.cpu().numpy()
    scale = np.abs(gw).max()
    assert np.abs(gg - gw).max() <= 1e-4 * scale + 1e-7
    # deterministic: the same call gives the same bits
    g2 = torch.empty_like(g)
    aclz.aclz_mlp_grad(dp, K, dx, dy, B, g2, loss, scratch)
    assert torch.equal(g, g2)


def test_adam_matches_oracle_over_steps():
    K, B = 12, 64
    p, x, y = _case(K, B, 7)
    dp, dx, dy = _dev(p), _dev(x), _dev(y, torch.int32)
    m = torch.zeros_like(dp)
    v = torch.zeros_like(dp)
    g = torch.empty_like(dp)
    loss = torch.empty(1, device="cuda")
    scratch = torch.empty(aclz.aclz_mlp_scratch_bytes(K, B), dtype=torch.uint8, device="cuda")
    pw, mw, vw = p.astype(np.float64), np.zeros(p.size), np.zeros(p.size)
    for t in range(1, 6):
        aclz.aclz_mlp_grad(dp, K, dx, dy, B, g, loss, scratch)
        # the oracle steps with the GPU's gradient so only the update rule is compared
        gn = g.cpu().numpy().astype(np.float64)
        aclz.aclz_mlp_adam(dp, m, v, g, K, t, 1e-3)
        pw, mw, vw = mlp.adam(pw, gn, mw, vw, t, lr=1e-3)
        assert np.abs(dp.cpu().numpy() - pw).max() < 1e-5
    assert np.allclose(m.cpu().numpy(), mw, rtol=1e-4, atol=1e-9)


@pytest.mark.parametrize("bs", [1000, 16384])
def test_block_features_match_oracle(bs):
    x = np.concatenate([synth.fastq(40_000, seed=1), synth.markov2(30_000, seed=2),
                        np.full(5000, 65, np.uint8), np.random.default_rng(3).integers(0, 256, 9_003).astype(np.uint8)])
    nb = -(-x.size // bs)
    dx = torch.from_numpy(x).cuda()
    f = torch.full((nb * 10,), float("nan"), device="cuda")
    aclz.aclz_block_features(dx, x.size, bs, f)
    got = f.view(nb, 10).cpu().numpy()
    want = mlp.raw_block_features(x, bs)
    assert np.allclose(got, want, rtol=1e-4, atol=2e-5)


def test_training_lowers_loss_and_learned_encode_is_exact():
    # small training set: two FASTQ-like and two Markov streams
    streams = [synth.fastq(1 << 20, seed=0x7A0000), synth.markov2(1 << 19, seed=0x7B0000),
               synth.fastq(1 << 20, seed=0x7A0001), synth.markov2(1 << 19, seed=0x7B0001)]
    feats, labels = [], []
    for s in streams:
        f, costs, ntok, ndef, ms = learned.label_data(s, threads=4)
        assert ndef.shape == ntok.shape and np.all(ndef <= ntok) and ms.shape == (learned.K,) and np.all(ms > 0)
        y, lam = learned.lagrange_labels(costs, ntok)
        assert f.shape == (y.size, learned.N_FEATURES) and lam >= 0
        # the labels meet the token target of their stream
        assert ntok[y, np.arange(y.size)].sum() <= learned.TOKEN_TARGET * ntok[learned.FALLBACK].sum() + 1e-9
        feats.append(f)
        labels.append(y)
    f = np.concatenate(feats)
    y = np.concatenate(labels)
    model = learned.Model()

    def xent(m):
        z = m.logits(f).astype(np.float64)
        z -= z.max(axis=1, keepdims=True)
        return float(np.mean(np.log(np.exp(z).sum(axis=1)) - z[np.arange(y.size), y]))

    model.mean, model.std = f.mean(axis=0), f.std(axis=0) + 1e-6
    before = xent(model)
    model.fit(f, y, steps=300, batch=128, lr=3e-3)
    assert xent(model) < before
    # evaluation stream (seed not used in training)
    x = np.concatenate([synth.fastq(1 << 20, seed=0x7A1000), synth.markov2(1 << 19, seed=0x7B1000)])
    c, k = learned.encode_learned(model, x)
    assert np.array_equal(oracle.decode(c), x)
    fb = learned.encode(x, learned.CANDIDATES[learned.FALLBACK])
    # the size-and-token check: no larger estimated size and no more tokens than 12/16/24/32
    assert learned.est_bytes(c) <= learned.est_bytes(fb)
    assert learned.read_tokens(c)[0].sum() <= learned.read_tokens(fb)[0].sum()
    h = aclz.aclz_upload(c, torch.cuda.current_stream())
    try:
        out = torch.empty(x.size + 16, dtype=torch.uint8, device="cuda")
        aclz.aclz_decode_all(h, out)
        torch.cuda.synchronize()
        assert np.array_equal(out[:x.size].cpu().numpy(), x)
    finally:
        aclz.aclz_free(h)
