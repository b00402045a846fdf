"""What the trained threshold network gains over the method without it: on
two held-out word-text streams (the serving corpus's generator, seeds
disjoint from training), the learned per-block thresholds, checked against
the plain encoder's ratio and measured decode speed, decode strictly
faster in total than the fixed 12/16/24/32 thresholds at an estimated size
no larger on each, with the network's picks kept on part of the blocks,
and the output exact.  The
network is trained here, on the GPU, from labels built from measured decode
times of the training streams; of several initialisations the one that
does best on a separate validation stream is kept."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, learned, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def model():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    aclz.lib()
    streams = ([synth.wordtext(4 << 20, seed=0x7C0000 + i, chunk_bytes=1 << 20) for i in range(3)] +
               [synth.fastq(4 << 20, seed=0x7A0000 + i) for i in range(2)] +
               [synth.markov2(2 << 20, seed=0x7B0000 + i) for i in range(2)])
    # model selection on a validation stream of its own, shaped like the
    # held-out stream below (neither is used for training)
    val = synth.wordtext(16 << 20, seed=0x7C0100, chunk_bytes=1 << 21)
    return learned.train_selected(streams, val, steps=800, log=lambda s: None)


def test_time_model_is_fitted_to_measured_decodes(model):
    a, b, c = model.time_coef
    assert a >= 0 and b >= 0 and c >= 0 and (a > 0 or b > 0)


def test_learned_thresholds_decode_faster_at_no_larger_size(model):
    # two held-out streams, judged together: total decode time of the
    # learned encodes against the fixed ones, sizes stream by stream
    tl = tf = 0.0
    kept = []
    for seed in (0x7C1000, 0x7C1001):
        x = synth.wordtext(16 << 20, seed=seed, chunk_bytes=1 << 21)
        fb = learned.encode(x, learned.CANDIDATES[learned.FALLBACK])
        ms = lambda c: x.size / learned.decode_gbs(c, x.size, reps=7)[0] / 1e6
        c, k = learned.encode_learned(model, x, fb=fb, time_coef=model.time_coef, judge=ms)
        kept.append(float(np.mean(k != learned.FALLBACK)))
        assert learned.est_bytes(c) <= learned.est_bytes(fb)
        gl, out = learned.decode_gbs(c, x.size, reps=9)
        assert np.array_equal(out.cpu().numpy(), x)
        assert np.array_equal(oracle.decode(c), x)
        gf, _ = learned.decode_gbs(fb, x.size, reps=9)
        tl += x.size / gl
        tf += x.size / gf
    assert max(kept) > 0.02, f"the check put (nearly) every block back to 12/16/24/32: kept {kept}"
    # strictly faster in total (the gain varies with the training run: from
    # under 1% to about 30% on these streams)
    assert tf > tl, f"learned {tl:.3g} vs fixed {tf:.3g} (decode time units), kept {kept}"
