"""Serving loop: Poisson-arriving range requests, admitted by memory and
batched continuously; every result equals the corpus slice, and equals the
same request decoded alone."""
import numpy as np
import pytest

from paper_2607_18541_gb300 import aclz, serve, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    aclz.lib()


@pytest.mark.parametrize("budget", [1 << 30, 6 << 20])
def test_results_in_the_mix_equal_slices_and_alone(budget):
    total = 24 << 20
    x, c = serve.build_corpus(total, block_size=1 << 14)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        arr, st, sz = synth.requests(150, 3000.0, 16 << 10, 4 << 20, total, seed=99)
        srv = serve.Server(h, budget, max_inflight=32, n_streams=3, max_batch=16)
        lat, span, outs = srv.run(arr, st, sz, keep_outputs=True)
        assert len(outs) == 150 and np.all(np.isfinite(lat)) and np.all(lat >= 0)
        for i in range(150):
            lo, n = int(st[i]), int(sz[i])
            assert np.array_equal(outs[i], x[lo:lo + n]), i
        for i in (0, 7, 149):
            lo, n = int(st[i]), int(sz[i])
            o = torch.empty((n + 15) // 16 * 16, dtype=torch.uint8, device="cuda")
            aclz.aclz_decode_range(h, lo, lo + n, o, stream=s)
            assert np.array_equal(o[:n].cpu().numpy(), outs[i])
        assert aclz.aclz_device_status(h, s) == 0
    finally:
        aclz.aclz_free(h)
