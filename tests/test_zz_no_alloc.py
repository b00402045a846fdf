"""The allocation-free FNV entry point, for callers that must not allocate
device memory while hashing (a nearly full device, memory owned by an arena
or pool manager, a latency-critical path kept out of the CUDA allocator).

It must give the same hash as the allocating aclz_fnv, call after call,
because its fixed scratch array is shared and keeps the previous call's
contents.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2607_18541_gb300 import aclz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _c_abi_fnv(name, t, n, stream):
    out = ctypes.c_uint64(0)
    rc = getattr(aclz.lib(), name)(ctypes.c_void_p(t.data_ptr()), ctypes.c_uint64(n),
                                   ctypes.byref(out), ctypes.c_void_p(stream.cuda_stream))
    return rc, int(out.value)


def test_noalloc_fnv_matches_allocating_fnv_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    s = torch.cuda.current_stream()
    rng = np.random.default_rng(2024)
    # two calls in a row on different contents and sizes: the second must
    # not see anything left over from the first
    for n in ((5 << 20) + 77, 300_001):
        x = torch.from_numpy(np.frombuffer(rng.bytes(n), dtype=np.uint8).copy()).cuda()
        rc_a, h_a = _c_abi_fnv("aclz_fnv_noalloc", x, n, s)
        rc_b, h_b = _c_abi_fnv("aclz_fnv", x, n, s)
        assert rc_a == aclz.ACLZ_OK and rc_b == aclz.ACLZ_OK
        assert h_a == h_b


def test_noalloc_fnv_rejects_inputs_beyond_its_fixed_limit():
    s = torch.cuda.current_stream()
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc, _ = _c_abi_fnv("aclz_fnv_noalloc", x, (4 << 30) + 1, s)
    assert rc == aclz.ACLZ_E_CAPACITY
