"""Thin ctypes binding of libaclz.so (include/aclz.h), same names as the
C ABI.  Argument marshalling only: every decode step runs in the library's
CUDA kernels.  Device buffers may be given as torch CUDA tensors or raw
integer pointers; streams as torch.cuda.Stream, raw handles or None.

There is no fallback: if libaclz.so is missing or fails to load, every call
raises ``AclzError``.  Build it with ``paper_2607_18541_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaclz.so")
_lock = threading.Lock()
_lib = None

ACLZ_OK = 0
ACLZ_E_INVAL = -1
ACLZ_E_CORRUPT = -2
ACLZ_E_NOMEM = -3
ACLZ_E_CAPACITY = -4
ACLZ_E_CUDA = -5
ACLZ_E_TIMEOUT = -6
ACLZ_E_DEVICE = -7
ACLZ_E_UNSUPPORTED = -8
ACLZ_PRESET_BASE, ACLZ_PRESET_TUNED, ACLZ_PRESET_PUSH = 0, 1, 2
ACLZ_UPLOAD_FLATTEN = 1
ACLZ_MODE_WAVES, ACLZ_MODE_PERSISTENT, ACLZ_MODE_AUTO = 0, 1, 2
ACLZ_FLAG_STAGED, ACLZ_FLAG_REGISTERS = 1, 2


class AclzError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = aclz_strerror(code) if _lib is not None else str(code)
        if code == ACLZ_E_CUDA and _lib is not None:
            msg += f" (cudaError {_lib.aclz_last_cuda_error()})"
        super().__init__(f"{what}: {msg} ({code})")
        self.code = code


class aclz_encode_params(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_uint32), ("min_match", ctypes.c_uint8 * 4),
                ("chain_depth", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("window", ctypes.c_uint64)]


class aclz_info(ctypes.Structure):
    _fields_ = [("total_len", ctypes.c_uint64), ("n_tokens", ctypes.c_uint64),
                ("n_literals", ctypes.c_uint64), ("n_deferred", ctypes.c_uint64),
                ("block_size", ctypes.c_uint32), ("n_blocks", ctypes.c_uint32),
                ("n_waves", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("min_match", ctypes.c_uint8 * 4), ("reserved", ctypes.c_uint32)]


class aclz_range_req(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64), ("d_out", ctypes.c_void_p),
                ("seg_base", ctypes.c_uint64)]


class aclz_decode_cfg(ctypes.Structure):
    _fields_ = [("G", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


# (name, restype, argtypes)
_VP, _U64, _U32, _I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
_U8P = ctypes.POINTER(ctypes.c_uint8)
_U32P = ctypes.POINTER(ctypes.c_uint32)
_U64P = ctypes.POINTER(ctypes.c_uint64)
_SIGS = [
    ("aclz_encode_params_default", _I, [ctypes.POINTER(aclz_encode_params), _I]),
    ("aclz_encode_bound", _U64, [_U64, _U32]),
    ("aclz_encode", _I, [_VP, _U64, ctypes.POINTER(aclz_encode_params), _U8P, _I, _VP, _U64, _U64P]),
    ("aclz_pack", _I, [_U64, _U32, _U8P, _U32P, _U32P, _U32P, _U64P, _U64, _U8P, _U64, _VP, _U64, _U64P]),
    ("aclz_pack_bytes", _U64, [_U64, _U32, _U64, _U64]),
    ("aclz_container_info", _I, [_VP, _U64, ctypes.POINTER(aclz_info)]),
    ("aclz_upload", _I, [_VP, _U64, _VP, ctypes.POINTER(_VP)]),
    ("aclz_upload_ex", _I, [_VP, _U64, _U32, _VP, ctypes.POINTER(_VP)]),
    ("aclz_upload_acle", _I, [_VP, _U64, _U32, _VP, ctypes.POINTER(_VP)]),
    ("aclz_acle_bound", _I, [_VP, _U64, ctypes.POINTER(_U64)]),
    ("aclz_acle_encode", _I, [_VP, _U64, _I, _VP, _U64, ctypes.POINTER(_U64)]),
    ("aclz_free", _I, [_VP]),
    ("aclz_handle_info", _I, [_VP, ctypes.POINTER(aclz_info)]),
    ("aclz_wave_counts", _I, [_VP, _U64P, _U32]),
    ("aclz_tags", _I, [_VP, _U32P, _U64]),
    ("aclz_set_range_bytes", _I, [_VP, _U32, _VP]),
    ("aclz_flatten", _I, [_VP, _VP]),
    ("aclz_selftest_wait", _I, [_U32, _VP]),
    ("aclz_export", _I, [_VP, _VP, _U64, _U64P]),
    ("aclz_reshape", _I, [_VP, _U32, _VP]),
    ("aclz_decode_all", _I, [_VP, _VP, _U64, ctypes.POINTER(aclz_decode_cfg), _VP]),
    ("aclz_decode_all_ev", _I, [_VP, _VP, _U64, ctypes.POINTER(aclz_decode_cfg), _VP, _VP]),
    ("aclz_decode_plan", _I, [_VP, ctypes.POINTER(aclz_decode_cfg), ctypes.POINTER(aclz_decode_cfg), _U32P]),
    ("aclz_device_status", _I, [_VP, _VP]),
    ("aclz_fnv", _I, [_VP, _U64, _U64P, _VP]),
    ("aclz_decode_range", _I, [_VP, _U64, _U64, _VP, _VP]),
    ("aclz_ranges_scratch_bytes", _I, [_U32, _U64P]),
    ("aclz_decode_ranges", _I, [_VP, _U32, _U64P, _U64P, ctypes.POINTER(_VP), _VP, _U64, _VP]),
    ("aclz_decode_ranges_async", _I, [_VP, _U32, _VP, _VP]),
    ("aclz_batch_merge", _I, [_U32, ctypes.POINTER(_VP), _U64P, _VP, _U64, _U64P, _U64P]),
    ("aclz_graph_create", _I, [_VP, _VP, _U64, ctypes.POINTER(aclz_decode_cfg), _VP, ctypes.POINTER(_VP)]),
    ("aclz_graph_launch", _I, [_VP, _VP]),
    ("aclz_graph_free", _I, [_VP]),
    ("aclz_mlp_param_count", _U32, [_U32]),
    ("aclz_mlp_scratch_bytes", _U64, [_U32, _U32]),
    ("aclz_mlp_forward", _I, [_VP, _U32, _VP, _U32, _VP, _VP]),
    ("aclz_mlp_grad", _I, [_VP, _U32, _VP, _VP, _U32, _VP, _VP, _VP, _U64, _VP]),
    ("aclz_mlp_adam", _I, [_VP, _VP, _VP, _VP, _U32, _U32, ctypes.c_float, _VP]),
    ("aclz_block_features", _I, [_VP, _U64, _U32, _VP, _VP]),
    ("aclz_strerror", ctypes.c_char_p, [_I]),
    ("aclz_last_cuda_error", _I, []),
]
OPTIONAL_SIGS: list = [  # entry points added by later modules register here
    ("aclz_fnv_noalloc", _I, [_VP, _U64, _U64P, _VP]),
    ("aclz_upload_acle_ev", _I, [_VP, _U64, _U32, _VP, ctypes.POINTER(_VP), _VP, _VP]),
    ("aclz_encode_gpu", _I, [_VP, _U64, ctypes.POINTER(aclz_encode_params), _VP, _VP, _VP, _U64, _U64P]),
]


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise AclzError(ACLZ_E_UNSUPPORTED, f"libaclz.so not built at {LIB_PATH}")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in _SIGS + OPTIONAL_SIGS:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_names() -> list[str]:
    return [s[0] for s in _SIGS + OPTIONAL_SIGS]


def _ck(rc: int, what: str) -> int:
    if rc < 0:
        raise AclzError(int(rc), what)
    return rc


def _dptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _hptr(a: np.ndarray) -> int:
    return int(a.ctypes.data)


def _np_u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    return np.ascontiguousarray(x).view(np.uint8).reshape(-1)


# ------------------------------------------------------------------ encode

def aclz_strerror(code: int) -> str:
    return lib().aclz_strerror(code).decode()


def aclz_encode_params_default(preset: int = ACLZ_PRESET_BASE) -> aclz_encode_params:
    p = aclz_encode_params()
    _ck(lib().aclz_encode_params_default(ctypes.byref(p), preset), "aclz_encode_params_default")
    return p


def aclz_encode_bound(n: int, block_size: int) -> int:
    return int(lib().aclz_encode_bound(n, block_size))


def aclz_encode(src, params: aclz_encode_params, block_min_match=None, threads: int = 0) -> np.ndarray:
    x = _np_u8(src)
    cap = aclz_encode_bound(x.size, params.block_size)
    out = np.empty(cap, dtype=np.uint8)
    size = ctypes.c_uint64(0)
    bmm = None
    if block_min_match is not None:
        bmm = np.ascontiguousarray(block_min_match, dtype=np.uint8).reshape(-1)
    _ck(lib().aclz_encode(_hptr(x) if x.size else None, x.size, ctypes.byref(params),
                          None if bmm is None else bmm.ctypes.data_as(_U8P), threads, _hptr(out), cap,
                          ctypes.byref(size)), "aclz_encode")
    return out[:size.value]


def aclz_encode_gpu(src, params: aclz_encode_params, block_min_match=None, stream=None) -> np.ndarray:
    """aclz_encode with the greedy parse on the GPU: the same container."""
    x = _np_u8(src)
    bmm = None
    if block_min_match is not None:
        bmm = np.ascontiguousarray(block_min_match, dtype=np.uint8)
    size = ctypes.c_uint64(0)
    bp = _hptr(bmm) if bmm is not None else None
    _ck(lib().aclz_encode_gpu(_hptr(x), x.size, ctypes.byref(params), bp, _stream(stream), None, 0,
                              ctypes.byref(size)), "aclz_encode_gpu")
    out = np.empty(max(1, size.value), dtype=np.uint8)
    _ck(lib().aclz_encode_gpu(_hptr(x), x.size, ctypes.byref(params), bp, _stream(stream), _hptr(out), out.size,
                              ctypes.byref(size)), "aclz_encode_gpu")
    return out[:size.value]


def aclz_pack_bytes(total_len: int, block_size: int, n_tokens: int, n_literals: int) -> int:
    return int(lib().aclz_pack_bytes(total_len, block_size, n_tokens, n_literals))


def aclz_pack(total_len: int, block_size: int, min_match, blk_ntok, lit_len, match_len, src,
              literals) -> np.ndarray:
    blk = np.ascontiguousarray(blk_ntok, dtype=np.uint32)
    ll = np.ascontiguousarray(lit_len, dtype=np.uint32)
    ml = np.ascontiguousarray(match_len, dtype=np.uint32)
    sr = np.ascontiguousarray(src, dtype=np.uint64)
    lits = _np_u8(literals)
    mm = (ctypes.c_uint8 * 4)(*min_match)
    cap = aclz_pack_bytes(total_len, block_size, ll.size, lits.size)
    out = np.empty(cap, dtype=np.uint8)
    size = ctypes.c_uint64(0)
    _ck(lib().aclz_pack(total_len, block_size, mm, blk.ctypes.data_as(_U32P), ll.ctypes.data_as(_U32P),
                        ml.ctypes.data_as(_U32P), sr.ctypes.data_as(_U64P), ll.size,
                        lits.ctypes.data_as(_U8P) if lits.size else None, lits.size, _hptr(out), cap,
                        ctypes.byref(size)), "aclz_pack")
    return out[:size.value]


def aclz_container_info(buf) -> aclz_info:
    c = _np_u8(buf)
    info = aclz_info()
    _ck(lib().aclz_container_info(_hptr(c), c.size, ctypes.byref(info)), "aclz_container_info")
    return info


# ------------------------------------------------------------------ device

def aclz_upload(buf, stream=None, flags: int = 0) -> int:
    """Returns the handle as an integer; flags = ACLZ_UPLOAD_* (aclz_upload_ex)."""
    c = _np_u8(buf)
    h = ctypes.c_void_p(0)
    if flags:
        _ck(lib().aclz_upload_ex(_hptr(c), c.size, flags, _stream(stream), ctypes.byref(h)), "aclz_upload_ex")
    else:
        _ck(lib().aclz_upload(_hptr(c), c.size, _stream(stream), ctypes.byref(h)), "aclz_upload")
    return int(h.value)


def aclz_upload_acle(buf, stream=None, flags: int = 0) -> int:
    """Upload an entropy-coded (ACLE) container; its tiles are decoded on
    the GPU.  Returns the handle as an integer."""
    e = _np_u8(buf)
    h = ctypes.c_void_p(0)
    _ck(lib().aclz_upload_acle(_hptr(e), e.size, flags, _stream(stream), ctypes.byref(h)), "aclz_upload_acle")
    return int(h.value)


def aclz_acle_encode(buf, threads: int = 0) -> np.ndarray:
    """The entropy-coded (ACLE) form of a host v1 container."""
    c = _np_u8(buf)
    bound = ctypes.c_uint64(0)
    _ck(lib().aclz_acle_bound(_hptr(c), c.size, ctypes.byref(bound)), "aclz_acle_bound")
    out = np.empty(bound.value, dtype=np.uint8)
    size = ctypes.c_uint64(0)
    _ck(lib().aclz_acle_encode(_hptr(c), c.size, threads, _hptr(out), out.size, ctypes.byref(size)),
        "aclz_acle_encode")
    return out[:size.value]


def aclz_free(h: int) -> None:
    _ck(lib().aclz_free(h), "aclz_free")


def aclz_handle_info(h: int) -> aclz_info:
    info = aclz_info()
    _ck(lib().aclz_handle_info(h, ctypes.byref(info)), "aclz_handle_info")
    return info


def aclz_wave_counts(h: int) -> np.ndarray:
    nw = aclz_handle_info(h).n_waves
    out = np.zeros(max(1, nw), dtype=np.uint64)
    _ck(lib().aclz_wave_counts(h, out.ctypes.data_as(_U64P), nw), "aclz_wave_counts")
    return out[:nw]


def aclz_tags(h: int) -> np.ndarray:
    nt = aclz_handle_info(h).n_tokens
    out = np.zeros(max(1, nt), dtype=np.uint32)
    _ck(lib().aclz_tags(h, out.ctypes.data_as(_U32P), nt), "aclz_tags")
    return out[:nt]


def aclz_export(h: int) -> np.ndarray:
    """The handle's stream as a host container carrying its wave tags."""
    size = ctypes.c_uint64(0)
    _ck(lib().aclz_export(h, None, 0, ctypes.byref(size)), "aclz_export")
    out = np.empty(size.value, dtype=np.uint8)
    _ck(lib().aclz_export(h, _hptr(out), out.size, ctypes.byref(size)), "aclz_export")
    return out


def aclz_selftest_wait(spin_limit: int, stream=None) -> int:
    """Status of the bounded-wait self-test (ACLZ_E_TIMEOUT expected)."""
    return int(lib().aclz_selftest_wait(spin_limit, _stream(stream)))


def aclz_flatten(h: int, stream=None) -> None:
    _ck(lib().aclz_flatten(h, _stream(stream)), "aclz_flatten")


def aclz_reshape(h: int, rounds: int, stream=None) -> None:
    _ck(lib().aclz_reshape(h, rounds, _stream(stream)), "aclz_reshape")


def aclz_set_range_bytes(h: int, range_bytes: int, stream=None) -> None:
    _ck(lib().aclz_set_range_bytes(h, range_bytes, _stream(stream)), "aclz_set_range_bytes")


def aclz_decode_all(h: int, d_out, cap: int | None = None, G: int = 32,
                    mode: int = ACLZ_MODE_AUTO, ctas_per_sm: int = 0, flags: int = 0,
                    stream=None) -> None:
    if cap is None:
        cap = int(d_out.numel() * d_out.element_size())
    cfg = aclz_decode_cfg(G, mode, ctas_per_sm, flags)
    _ck(lib().aclz_decode_all(h, _dptr(d_out), cap, ctypes.byref(cfg), _stream(stream)), "aclz_decode_all")


def aclz_decode_plan(h: int, G: int = 32, mode: int = ACLZ_MODE_AUTO, ctas_per_sm: int = 0, flags: int = 0):
    """(resolved cfg as a dict, kernel launches per aclz_decode_all call)."""
    cfg = aclz_decode_cfg(G, mode, ctas_per_sm, flags)
    res = aclz_decode_cfg()
    n = ctypes.c_uint32(0)
    _ck(lib().aclz_decode_plan(h, ctypes.byref(cfg), ctypes.byref(res), ctypes.byref(n)), "aclz_decode_plan")
    return dict(G=res.G, mode=res.mode, ctas_per_sm=res.ctas_per_sm, flags=res.flags), int(n.value)


def aclz_decode_all_ev(h: int, d_out, phase_event, cap: int | None = None, G: int = 32,
                       mode: int = ACLZ_MODE_AUTO, ctas_per_sm: int = 0, flags: int = 0,
                       stream=None) -> None:
    """phase_event: a torch.cuda.Event (timing enabled) or a raw cudaEvent_t."""
    if cap is None:
        cap = int(d_out.numel() * d_out.element_size())
    ev = phase_event if isinstance(phase_event, int) else int(phase_event.cuda_event)
    if not ev:
        raise ValueError("phase_event has no CUDA event yet: record it once before passing it")
    cfg = aclz_decode_cfg(G, mode, ctas_per_sm, flags)
    _ck(lib().aclz_decode_all_ev(h, _dptr(d_out), cap, ctypes.byref(cfg), _stream(stream), ev),
        "aclz_decode_all_ev")


def aclz_device_status(h: int, stream=None) -> int:
    return _ck(lib().aclz_device_status(h, _stream(stream)), "aclz_device_status")


def aclz_decode_range(h: int, lo: int, hi: int, d_out, stream=None) -> None:
    _ck(lib().aclz_decode_range(h, lo, hi, _dptr(d_out), _stream(stream)), "aclz_decode_range")


def aclz_ranges_scratch_bytes(n_requests: int) -> int:
    out = ctypes.c_uint64(0)
    _ck(lib().aclz_ranges_scratch_bytes(n_requests, ctypes.byref(out)), "aclz_ranges_scratch_bytes")
    return int(out.value)


def aclz_decode_ranges(h: int, lo, hi, outs, d_scratch, scratch_cap: int | None = None, stream=None) -> None:
    n = len(lo)
    lo_a = np.ascontiguousarray(lo, dtype=np.uint64)
    hi_a = np.ascontiguousarray(hi, dtype=np.uint64)
    ptrs = (_VP * max(1, n))(*[_dptr(o) for o in outs])
    if scratch_cap is None:
        scratch_cap = int(d_scratch.numel() * d_scratch.element_size())
    _ck(lib().aclz_decode_ranges(h, n, lo_a.ctypes.data_as(_U64P), hi_a.ctypes.data_as(_U64P), ptrs,
                                 _dptr(d_scratch), scratch_cap, _stream(stream)), "aclz_decode_ranges")


def aclz_decode_ranges_async(h: int, n: int, reqs_ptr: int, stream=None) -> None:
    """reqs_ptr: address of n aclz_range_req in pinned host memory (32 B each:
    lo, hi, d_out, seg_base), kept alive until the launch completes."""
    _ck(lib().aclz_decode_ranges_async(h, n, reqs_ptr, _stream(stream)), "aclz_decode_ranges_async")


def aclz_batch_merge(containers):
    """Returns (merged container, per-stream output offsets)."""
    arrs = [_np_u8(c) for c in containers]
    n = len(arrs)
    ptrs = (_VP * n)(*[_hptr(a) if a.size else None for a in arrs])
    sizes = np.array([a.size for a in arrs], dtype=np.uint64)
    offs = np.zeros(n, dtype=np.uint64)
    need = ctypes.c_uint64(0)
    _ck(lib().aclz_batch_merge(n, ptrs, sizes.ctypes.data_as(_U64P), None, 0, ctypes.byref(need),
                               offs.ctypes.data_as(_U64P)), "aclz_batch_merge")
    out = np.empty(need.value, dtype=np.uint8)
    size = ctypes.c_uint64(0)
    _ck(lib().aclz_batch_merge(n, ptrs, sizes.ctypes.data_as(_U64P), _hptr(out), out.size, ctypes.byref(size),
                               offs.ctypes.data_as(_U64P)), "aclz_batch_merge")
    return out[:size.value], offs


def aclz_graph_create(h: int, d_out, cap: int | None = None, G: int = 32, mode: int = ACLZ_MODE_AUTO,
                      ctas_per_sm: int = 0, flags: int = 0, stream=None) -> int:
    if cap is None:
        cap = int(d_out.numel() * d_out.element_size())
    cfg = aclz_decode_cfg(G, mode, ctas_per_sm, flags)
    g = ctypes.c_void_p(0)
    _ck(lib().aclz_graph_create(h, _dptr(d_out), cap, ctypes.byref(cfg), _stream(stream), ctypes.byref(g)),
        "aclz_graph_create")
    return int(g.value)


def aclz_graph_launch(g: int, stream=None) -> None:
    _ck(lib().aclz_graph_launch(g, _stream(stream)), "aclz_graph_launch")


def aclz_graph_free(g: int) -> None:
    _ck(lib().aclz_graph_free(g), "aclz_graph_free")


def aclz_mlp_param_count(K: int) -> int:
    return int(lib().aclz_mlp_param_count(K))


def aclz_mlp_scratch_bytes(K: int, batch: int) -> int:
    return int(lib().aclz_mlp_scratch_bytes(K, batch))


def aclz_mlp_forward(d_params, K: int, d_x, batch: int, d_logits, stream=None) -> None:
    _ck(lib().aclz_mlp_forward(_dptr(d_params), K, _dptr(d_x), batch, _dptr(d_logits), _stream(stream)),
        "aclz_mlp_forward")


def aclz_mlp_grad(d_params, K: int, d_x, d_y, batch: int, d_grad, d_loss, d_scratch, scratch_bytes=None,
                  stream=None) -> None:
    if scratch_bytes is None:
        scratch_bytes = int(d_scratch.numel() * d_scratch.element_size())
    _ck(lib().aclz_mlp_grad(_dptr(d_params), K, _dptr(d_x), _dptr(d_y), batch, _dptr(d_grad), _dptr(d_loss),
                            _dptr(d_scratch), scratch_bytes, _stream(stream)), "aclz_mlp_grad")


def aclz_mlp_adam(d_params, d_m, d_v, d_grad, K: int, step: int, lr: float, stream=None) -> None:
    _ck(lib().aclz_mlp_adam(_dptr(d_params), _dptr(d_m), _dptr(d_v), _dptr(d_grad), K, step, lr, _stream(stream)),
        "aclz_mlp_adam")


def aclz_block_features(d_x, n: int, block_size: int, d_feat, stream=None) -> None:
    _ck(lib().aclz_block_features(_dptr(d_x), n, block_size, _dptr(d_feat), _stream(stream)),
        "aclz_block_features")


def aclz_fnv(d_buf, n: int | None = None, stream=None) -> int:
    if n is None:
        n = int(d_buf.numel() * d_buf.element_size())
    out = ctypes.c_uint64(0)
    _ck(lib().aclz_fnv(_dptr(d_buf), n, ctypes.byref(out), _stream(stream)), "aclz_fnv")
    return int(out.value)


def aclz_fnv_noalloc(d_buf, n: int | None = None, stream=None) -> int:
    """aclz_fnv without device allocation (fixed 4 GiB limit, calls must not
    overlap on the GPU); see include/aclz.h."""
    if n is None:
        n = int(d_buf.numel() * d_buf.element_size())
    out = ctypes.c_uint64(0)
    _ck(lib().aclz_fnv_noalloc(_dptr(d_buf), n, ctypes.byref(out), _stream(stream)), "aclz_fnv_noalloc")
    return int(out.value)
