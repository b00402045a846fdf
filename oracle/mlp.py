"""CPU oracle (float64 numpy) for the learned-threshold network and its block
features (test infrastructure only).

The paper has no learned component; its lever (Sec. IV) is a fixed
minimum-match-length vector by distance class.  The network here picks one
of K candidate vectors per block from block statistics.  This module states,
plainly, what the GPU kernels compute:

  h1 = relu(x W1 + b1)      x: [B, 24], W1: [24, 64]
  h2 = relu(h1 W2 + b2)     W2: [64, 64]
  z  = h2 W3 + b3           W3: [64, K]
  loss = mean_b( -log softmax(z_b)[y_b] )

with gradients by the chain rule and Adam (Kingma & Ba, 2015) with bias
correction.  Parameters are one flat float vector in the order W1, b1, W2,
b2, W3, b3 (row-major).  Pinned by central finite differences and by closed
forms in tests/test_mlp_oracle.py.
"""
from __future__ import annotations

import numpy as np

D, H = 24, 64


def shapes(K: int):
    return [(D, H), (H,), (H, H), (H,), (H, K), (K,)]


def n_params(K: int) -> int:
    return sum(int(np.prod(s)) for s in shapes(K))


def unpack(p: np.ndarray, K: int):
    out, o = [], 0
    for s in shapes(K):
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    return out


def init(K: int, seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in shapes(K):
        if len(s) == 2:
            parts.append(rng.standard_normal(s) * np.sqrt(2.0 / s[0]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate([q.reshape(-1) for q in parts])


def forward(p, x, K):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(p, dtype=np.float64), K)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3 + b3
    return z, (x, a1, h1, a2, h2)


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss(p, x, y, K) -> float:
    z, _ = forward(p, x, K)
    pr = softmax(z)
    return float(-np.mean(np.log(pr[np.arange(len(y)), y])))


def grads(p, x, y, K):
    """(loss, flat gradient) by backpropagation."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(p, dtype=np.float64), K)
    z, (x, a1, h1, a2, h2) = forward(p, x, K)
    B = x.shape[0]
    pr = softmax(z)
    L = float(-np.mean(np.log(pr[np.arange(B), y])))
    dz = pr.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    gW3 = h2.T @ dz
    gb3 = dz.sum(axis=0)
    dh2 = dz @ W3.T
    da2 = dh2 * (a2 > 0)
    gW2 = h1.T @ da2
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2.T
    da1 = dh1 * (a1 > 0)
    gW1 = x.T @ da1
    gb1 = da1.sum(axis=0)
    g = np.concatenate([q.reshape(-1) for q in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return L, g


def adam(p, g, m, v, step: int, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (step counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------ features

RAW_FEATURES = 10


def raw_block_features(x: np.ndarray, block_size: int) -> np.ndarray:
    """Per-block byte statistics, [n_blocks, 10]:
    0 order-0 entropy / 8, 1 distinct byte values / 256, 2 fraction of
    positions equal to the previous byte, 3 and 4: 1 - (estimated distinct
    4-grams and 8-grams) / positions, by linear counting over a 65536-bit
    map of a multiplicative hash, 5..9 fractions of digits, lowercase,
    uppercase, space/punctuation (0x20..0x2F, 0x3A..0x40, 0x5B..0x60,
    0x7B..0x7E) and all other bytes."""
    x = np.asarray(x, dtype=np.uint8)
    n = x.size
    nb = (n + block_size - 1) // block_size
    out = np.zeros((nb, RAW_FEATURES))
    for b in range(nb):
        s = x[b * block_size:min(n, (b + 1) * block_size)].astype(np.uint64)
        m = s.size
        cnt = np.bincount(s.astype(np.int64), minlength=256).astype(np.float64)
        pr = cnt[cnt > 0] / m
        out[b, 0] = -(pr * np.log2(pr)).sum() / 8.0
        out[b, 1] = np.count_nonzero(cnt) / 256.0
        out[b, 2] = np.count_nonzero(s[1:] == s[:-1]) / m if m > 1 else 0.0
        for f, k in ((3, 4), (4, 8)):
            if m >= k:
                key = np.zeros(m - k + 1, dtype=np.uint64)
                for j in range(k):
                    key |= s[j:m - k + 1 + j] << np.uint64(8 * j)
                hsh = ((key * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(48)).astype(np.int64)
                bits = np.zeros(65536, dtype=bool)
                bits[hsh] = True
                z = 65536 - np.count_nonzero(bits)
                est = -65536.0 * np.log(max(z, 1) / 65536.0)
                out[b, f] = 1.0 - min(est, m - k + 1) / (m - k + 1)
        c = s.astype(np.int64)
        dig = (c >= 0x30) & (c <= 0x39)
        low = (c >= 0x61) & (c <= 0x7A)
        up = (c >= 0x41) & (c <= 0x5A)
        pun = ((c >= 0x20) & (c <= 0x2F)) | ((c >= 0x3A) & (c <= 0x40)) | ((c >= 0x5B) & (c <= 0x60)) | \
              ((c >= 0x7B) & (c <= 0x7E))
        out[b, 5] = dig.mean()
        out[b, 6] = low.mean()
        out[b, 7] = up.mean()
        out[b, 8] = pun.mean()
        out[b, 9] = 1.0 - out[b, 5:9].sum()
    return out
