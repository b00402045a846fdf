"""Pins of the learned-threshold oracle (oracle/mlp.py) against facts that do
not come from its own formulas: central finite differences of the loss,
closed forms of softmax cross-entropy and of Adam's first step, and block
statistics whose values follow from the definition of each feature."""
import numpy as np
import pytest

from oracle import mlp


def _net(K=5, B=7, seed=3):
    rng = np.random.default_rng(seed)
    p = mlp.init(K, seed) + rng.standard_normal(mlp.n_params(K)) * 0.05
    x = rng.standard_normal((B, mlp.D))
    y = rng.integers(0, K, B)
    return p, x, y


def test_param_count_matches_layer_shapes():
    assert mlp.n_params(12) == 24 * 64 + 64 + 64 * 64 + 64 + 64 * 12 + 12
    assert mlp.n_params(3) == 24 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3


def test_gradient_equals_central_finite_differences():
    K = 4
    p, x, y = _net(K)
    L, g = mlp.grads(p, x, y, K)
    assert L == pytest.approx(mlp.loss(p, x, y, K), rel=1e-12)
    rng = np.random.default_rng(9)
    # every bias and a sample of each weight matrix
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mlp.shapes(K)])
    idx = []
    for a, b in zip(offs[:-1], offs[1:]):
        idx += list(rng.choice(np.arange(a, b), size=min(40, b - a), replace=False))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, x, y, K) - mlp.loss(p - e, x, y, K)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_uniform_logits_give_log_K_and_softmax_gradient():
    K, B = 6, 5
    p, x, y = _net(K, B)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, K)
    W3[:] = 0.0
    b3[:] = 0.0
    L, g = mlp.grads(p, x, y, K)
    assert L == pytest.approx(np.log(K), rel=1e-12)
    gb3 = mlp.unpack(g, K)[5]
    # d loss / d b3_k = mean_b (1/K - [y_b = k])
    want = np.full(K, 1.0 / K) - np.bincount(y, minlength=K) / B
    assert np.allclose(gb3, want, atol=1e-14)
    # zero last layer: nothing flows back to the hidden layers
    for q in mlp.unpack(g, K)[:4]:
        assert np.all(q == 0.0)


def test_output_bias_gradient_sums_to_zero():
    p, x, y = _net(7, 11)
    _, g = mlp.grads(p, x, y, 7)
    assert abs(mlp.unpack(g, 7)[5].sum()) < 1e-14


def test_loss_is_shift_invariant_in_output_bias():
    K = 5
    p, x, y = _net(K)
    q = p.copy()
    mlp.unpack(q, K)[5][:] += 3.25
    assert mlp.loss(q, x, y, K) == pytest.approx(mlp.loss(p, x, y, K), rel=1e-12)


def test_adam_first_step_is_sign_step():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(100)
    g = rng.standard_normal(100)
    m = np.zeros(100)
    v = np.zeros(100)
    p1, m1, v1 = mlp.adam(p, g, m, v, 1, lr=0.01)
    # m-hat = g, v-hat = g^2 after one step, so the update is lr * g / (|g| + eps)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g)
    assert np.allclose(v1, 0.001 * g * g)


def test_adam_constant_gradient_keeps_unit_steps():
    # with a constant gradient both bias-corrected moments equal g and g^2
    p = np.array([1.0, -2.0])
    g = np.array([0.5, -4.0])
    m = np.zeros(2)
    v = np.zeros(2)
    for t in range(1, 20):
        p, m, v = mlp.adam(p, g, m, v, t, lr=0.1)
    assert np.allclose(p, np.array([1.0, -2.0]) - 19 * 0.1 * np.sign(g), atol=1e-7)


def test_training_reduces_loss_on_separable_data():
    K, B = 3, 96
    rng = np.random.default_rng(0)
    y = rng.integers(0, K, B)
    x = rng.standard_normal((B, mlp.D)) * 0.1
    x[np.arange(B), y] += 2.0
    p = mlp.init(K, 5)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = mlp.loss(p, x, y, K)
    for t in range(1, 151):
        _, g = mlp.grads(p, x, y, K)
        p, m, v = mlp.adam(p, g, m, v, t, lr=3e-3)
    assert mlp.loss(p, x, y, K) < 0.1 * L0


# ------------------------------------------------------------ features

def test_features_of_a_constant_block():
    m = 4096
    f = mlp.raw_block_features(np.full(m, ord("a"), np.uint8), m)[0]
    assert f[0] == 0.0                       # one symbol: zero entropy
    assert f[1] == 1 / 256
    assert f[2] == pytest.approx((m - 1) / m)
    # one distinct n-gram: linear counting estimates -65536 ln(65535/65536) ~ 1
    for col, k in ((3, 4), (4, 8)):
        est = -65536.0 * np.log(65535 / 65536)
        assert f[col] == pytest.approx(1 - est / (m - k + 1), rel=1e-12)
    assert f[6] == 1.0 and f[5] == f[7] == f[8] == f[9] == 0.0


def test_features_of_all_byte_values():
    x = np.tile(np.arange(256, dtype=np.uint8), 16)
    f = mlp.raw_block_features(x, x.size)[0]
    assert f[0] == pytest.approx(1.0)        # 8 bits per byte / 8
    assert f[1] == 1.0
    assert f[2] == 0.0
    assert f[5] == pytest.approx(10 / 256)
    assert f[6] == pytest.approx(26 / 256) and f[7] == pytest.approx(26 / 256)
    assert f[8] == pytest.approx(33 / 256)   # 95 printable 0x20..0x7E minus 62 alphanumerics
    assert f[9] == pytest.approx(1 - 95 / 256)
    # 256 distinct 4-grams among 4093 positions
    assert f[3] == pytest.approx(1 - 256 / 4093, abs=3e-3)


def test_features_of_digits_and_random_bytes():
    x = np.frombuffer(b"0123456789" * 400, np.uint8)
    f = mlp.raw_block_features(x, x.size)[0]
    assert f[0] == pytest.approx(np.log2(10) / 8)
    assert f[5] == 1.0
    # random bytes: almost every 4-gram is new
    r = np.random.default_rng(4).integers(0, 256, 16384).astype(np.uint8)
    g = mlp.raw_block_features(r, r.size)[0]
    assert abs(g[3]) < 0.02 and abs(g[4]) < 0.02
    assert g[0] > 0.98


def test_features_split_blocks_and_ragged_tail():
    rng = np.random.default_rng(2)
    x = rng.integers(0, 256, 3 * 1000 + 17).astype(np.uint8)
    f = mlp.raw_block_features(x, 1000)
    assert f.shape == (4, 10)
    for b in range(4):
        one = mlp.raw_block_features(x[b * 1000:(b + 1) * 1000], 1000)[0]
        assert np.array_equal(f[b], one)
    # a one-byte tail: no n-grams, no repeats
    t = mlp.raw_block_features(np.array([7], np.uint8), 1)[0]
    assert t[2] == 0.0 and t[3] == 0.0 and t[4] == 0.0 and t[9] == 1.0
