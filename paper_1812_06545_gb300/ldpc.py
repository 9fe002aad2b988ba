"""Thin Python binding of the C ABI in include/ldpc.h (argument marshalling only).

Every decoding step runs in the CUDA library ``libldpc_gb300.so``; this module only turns
torch tensors / numpy arrays into pointers and CUDA streams into handles.  There is no
fallback: if the library is missing, every call raises.

The functions carry the C names (``ldpc_code_create``, ``ldpc_decode_batch``, ...);
``Code``, ``default_params`` and ``decode`` are small conveniences on top of them.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libldpc_gb300.so")

LDPC_OK, LDPC_EINVAL, LDPC_ENOMEM, LDPC_ECUDA, LDPC_EBUSY, LDPC_ETIMEDOUT, LDPC_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
LDPC_SCHED_FLOODING, LDPC_SCHED_LAYERED = 0, 1
LDPC_ALGO_SPA, LDPC_ALGO_NMS = 0, 1
LDPC_MSG_F32, LDPC_MSG_F16, LDPC_MSG_I8 = 0, 1, 2
LDPC_LLR_F32, LDPC_LLR_I8 = 0, 1
LDPC_IMPL_AUTO, LDPC_IMPL_PLAIN, LDPC_IMPL_STREAMING, LDPC_IMPL_CLUSTER = 0, 1, 2, 3
FAMILIES = {"interleave": 0, "check_node": 1, "variable_node": 2, "deinterleave": 3, "layered": 4,
            "plain_check_node": 5, "plain_variable_node": 6, "slots": 7, "layered_spa": 8}


class LdpcError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what} failed with status {status}: {msg}")
        self.status = status


class Request(C.Structure):
    _fields_ = [("code", C.c_void_p), ("llr_dev", C.c_void_p), ("n_cw", C.c_int64), ("bits_dev", C.c_void_p),
                ("iters_dev", C.c_void_p), ("app_dev", C.c_void_p)]


class SessionConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_inflight", C.c_int32), ("max_batch", C.c_int32),
                ("start_paused", C.c_int32), ("fail_alloc_after", C.c_int32), ("reserved", C.c_int32 * 4)]


class SessionStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("cancelled", C.c_int64),
                ("queued", C.c_int64), ("launches", C.c_int64), ("budget_bytes", C.c_size_t),
                ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t)]


LDPC_REQ_QUEUED, LDPC_REQ_RUNNING, LDPC_REQ_DONE, LDPC_REQ_FAILED, LDPC_REQ_CANCELLED = 0, 1, 2, 3, 4


class DecodeParams(C.Structure):
    _fields_ = [("sched", C.c_int32), ("algo", C.c_int32), ("msg", C.c_int32), ("max_iter", C.c_int32),
                ("early_exit", C.c_int32), ("phi_clamp", C.c_float), ("nms_alpha_num", C.c_int32),
                ("nms_alpha_shift", C.c_int32), ("msg_sat", C.c_int32), ("app_sat", C.c_int32),
                ("llr_scale", C.c_float), ("impl", C.c_int32), ("reserved", C.c_int32 * 4)]


_lib = None


def lib():
    """Load the CUDA library (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() or "
                               "python -m paper_1812_06545_gb300._build")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        sig = {
            "ldpc_default_params": [vp],
            "ldpc_code_create": [vp, i32, i32, i32, vp],
            "ldpc_code_info": [vp, vp, vp, vp, vp],
            "ldpc_workspace_size": [vp, vp, i64, vp],
            "ldpc_decode_batch": [vp, vp, vp, i32, i64, vp, vp, vp, vp, sz, vp],
            "ldpc_decode_host": [vp, vp, vp, i64, vp, vp, i32, i64],
            "ldpc_decode_batch_static": [vp, vp, vp, i64, vp, vp, vp, vp],
            "ldpc_decode_multi": [vp, i32, vp, i32, vp, sz, vp],
            "ldpc_multi_workspace_size": [vp],
            "ldpc_autotune": [vp, vp, vp, i32, i64, vp, vp, vp],
            "ldpc_session_default_config": [vp],
            "ldpc_session_create": [vp, vp],
            "ldpc_session_submit": [vp, vp, vp, vp, i64, vp, vp, vp],
            "ldpc_session_poll": [vp, C.c_uint64, vp, vp],
            "ldpc_session_wait": [vp, C.c_uint64, C.c_double, vp],
            "ldpc_session_cancel": [vp, C.c_uint64],
            "ldpc_session_pause": [vp, i32],
            "ldpc_session_stats_get": [vp, vp],
            "ldpc_sfu_throughput": [vp, vp, vp],
            "ldpc_stream_check": [vp, vp],
            "ldpc_profile_enable": [i32],
            "ldpc_profile_read": [i32, vp, vp],
            "ldpc_profile_reset": [],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.ldpc_session_destroy.argtypes = [vp]
        L.ldpc_session_destroy.restype = None
        L.ldpc_code_destroy.argtypes = [vp]
        L.ldpc_code_destroy.restype = None
        L.ldpc_release_host_buffers.argtypes = []
        L.ldpc_release_host_buffers.restype = None
        L.ldpc_last_error.argtypes = []
        L.ldpc_last_error.restype = C.c_char_p
        L.ldpc_launch_count.argtypes = []
        L.ldpc_launch_count.restype = C.c_int64
        L.ldpc_launch_count_reset.argtypes = []
        L.ldpc_launch_count_reset.restype = None
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != LDPC_OK:
        raise LdpcError(st, what, lib().ldpc_last_error().decode())


def _ptr(x):
    """Device or host address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


# ------------------------------------------------------------------ C names

def ldpc_default_params(**overrides) -> DecodeParams:
    p = DecodeParams()
    _check(lib().ldpc_default_params(C.byref(p)), "ldpc_default_params")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown decode parameter {k}")
        setattr(p, k, v)
    return p


def ldpc_code_create(base, Z: int) -> int:
    b = np.ascontiguousarray(base, dtype=np.int32)
    h = C.c_void_p()
    _check(lib().ldpc_code_create(b.ctypes.data, b.shape[0], b.shape[1], int(Z), C.byref(h)), "ldpc_code_create")
    return h.value


def ldpc_code_destroy(handle: int) -> None:
    lib().ldpc_code_destroy(handle)


def ldpc_code_info(handle: int):
    N, K, M, E = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64()
    _check(lib().ldpc_code_info(handle, C.byref(N), C.byref(K), C.byref(M), C.byref(E)), "ldpc_code_info")
    return N.value, K.value, M.value, E.value


def ldpc_workspace_size(handle: int, params: DecodeParams, n_cw: int) -> int:
    b = C.c_size_t()
    _check(lib().ldpc_workspace_size(handle, C.byref(params), int(n_cw), C.byref(b)), "ldpc_workspace_size")
    return b.value


def ldpc_decode_batch(handle: int, params: DecodeParams, llr, llr_type: int, n_cw: int, bits, iters, app=None,
                      workspace=None, workspace_bytes: int = 0, stream=None) -> None:
    _check(lib().ldpc_decode_batch(handle, C.byref(params), _ptr(llr), int(llr_type), int(n_cw), _ptr(bits),
                                   _ptr(iters), _ptr(app), _ptr(workspace), int(workspace_bytes), _stream(stream)),
           "ldpc_decode_batch")


def ldpc_decode_multi(requests, params: DecodeParams, llr_type: int = LDPC_LLR_F32, workspace=None,
                      workspace_bytes: int = 0, stream=None) -> None:
    """requests: sequence of (code_handle, llr, n_cw, bits, iters, app_or_None)."""
    arr = (Request * max(1, len(requests)))()
    for i, (h, llr, n, bits, iters, app) in enumerate(requests):
        arr[i] = Request(h, _ptr(llr), int(n), _ptr(bits), _ptr(iters), _ptr(app))
    _check(lib().ldpc_decode_multi(arr, len(requests), C.byref(params), int(llr_type), _ptr(workspace),
                                   int(workspace_bytes), _stream(stream)), "ldpc_decode_multi")


def ldpc_autotune(handle: int, params: DecodeParams, llr, llr_type: int, n_cw: int, stream=None):
    """Time the candidate schedules on a device sample; returns (choice, [ms per candidate])."""
    choice = C.c_int32()
    ms = (C.c_float * 3)()
    _check(lib().ldpc_autotune(handle, C.byref(params), _ptr(llr), int(llr_type), int(n_cw), _stream(stream),
                               C.byref(choice), ms), "ldpc_autotune")
    return choice.value, list(ms)


def ldpc_session_default_config(**overrides) -> SessionConfig:
    c = SessionConfig()
    _check(lib().ldpc_session_default_config(C.byref(c)), "ldpc_session_default_config")
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def ldpc_session_create(cfg: SessionConfig) -> int:
    h = C.c_void_p()
    _check(lib().ldpc_session_create(C.byref(cfg), C.byref(h)), "ldpc_session_create")
    return h.value


def ldpc_session_submit(sess: int, code_handle: int, params: DecodeParams, llr_host, n_cw: int, bits_host,
                        iters_host=None) -> int:
    rid = C.c_uint64()
    _check(lib().ldpc_session_submit(sess, code_handle, C.byref(params), _ptr(llr_host), int(n_cw), _ptr(bits_host),
                                     _ptr(iters_host), C.byref(rid)), "ldpc_session_submit")
    return rid.value


def ldpc_session_poll(sess: int, rid: int):
    """-> (state, status, latency_s); status/latency only meaningful for finished states."""
    st, lat = C.c_int32(), C.c_double()
    rc = lib().ldpc_session_poll(sess, rid, C.byref(st), C.byref(lat))
    if st.value < LDPC_REQ_DONE and rc != LDPC_OK:
        _check(rc, "ldpc_session_poll")
    return st.value, rc, lat.value


def ldpc_session_wait(sess: int, rid: int, timeout_s: float) -> tuple[int, float]:
    """-> (status, latency_s); status LDPC_ETIMEDOUT if not finished in time."""
    lat = C.c_double()
    rc = lib().ldpc_session_wait(sess, rid, float(timeout_s), C.byref(lat))
    return rc, lat.value


def ldpc_session_cancel(sess: int, rid: int) -> int:
    return lib().ldpc_session_cancel(sess, rid)


def ldpc_session_pause(sess: int, paused: bool) -> None:
    _check(lib().ldpc_session_pause(sess, 1 if paused else 0), "ldpc_session_pause")


def ldpc_session_stats_get(sess: int) -> SessionStats:
    st = SessionStats()
    _check(lib().ldpc_session_stats_get(sess, C.byref(st)), "ldpc_session_stats_get")
    return st


def ldpc_session_destroy(sess: int) -> None:
    lib().ldpc_session_destroy(sess)


def ldpc_sfu_throughput(stream=None) -> tuple[float, float]:
    """Measured (ex2, lg2) special-function operations per second of the current device."""
    a, b = C.c_double(), C.c_double()
    _check(lib().ldpc_sfu_throughput(C.byref(a), C.byref(b), _stream(stream)), "ldpc_sfu_throughput")
    return a.value, b.value


def ldpc_multi_workspace_size() -> int:
    b = C.c_size_t()
    _check(lib().ldpc_multi_workspace_size(C.byref(b)), "ldpc_multi_workspace_size")
    return b.value


LDPC_STATIC_SCRATCH_BYTES = 32 << 20


def ldpc_decode_batch_static(handle: int, params: DecodeParams, llr, n_cw: int, bits, iters, app=None,
                             stream=None) -> None:
    """Flooding decode whose scratch is the library's fixed device array (no allocation).

    For callers that must not allocate device memory while decoding; batches needing more
    than LDPC_STATIC_SCRATCH_BYTES of scratch are rejected, and calls that overlap on the
    GPU share (and corrupt) the one array.  The first call on a device looks up the array's
    address, so make it before any stream capture."""
    _check(lib().ldpc_decode_batch_static(handle, C.byref(params), _ptr(llr), int(n_cw), _ptr(bits), _ptr(iters),
                                          _ptr(app), _stream(stream)), "ldpc_decode_batch_static")


def ldpc_decode_host(handle: int, params: DecodeParams, llr_host, n_cw: int, bits_host, iters_host=None,
                     n_streams: int = 1, chunk_cw: int = 0) -> None:
    _check(lib().ldpc_decode_host(handle, C.byref(params), _ptr(llr_host), int(n_cw), _ptr(bits_host),
                                  _ptr(iters_host), int(n_streams), int(chunk_cw)), "ldpc_decode_host")


def ldpc_stream_check(stream=None) -> int:
    """Take the device's input status word after the work queued on ``stream``; returns the
    flag bits (raises LdpcError with LDPC_EINVAL when a bit was set)."""
    f = C.c_uint32()
    _check(lib().ldpc_stream_check(_stream(stream), C.byref(f)), "ldpc_stream_check")
    return f.value


def ldpc_stream_flags(stream=None) -> int:
    """Like ldpc_stream_check, but returns the flag bits instead of raising on them."""
    f = C.c_uint32()
    st = lib().ldpc_stream_check(_stream(stream), C.byref(f))
    if st not in (LDPC_OK, LDPC_EINVAL):
        _check(st, "ldpc_stream_check")
    return f.value


def ldpc_release_host_buffers() -> None:
    lib().ldpc_release_host_buffers()


def ldpc_profile_enable(on: bool) -> None:
    _check(lib().ldpc_profile_enable(1 if on else 0), "ldpc_profile_enable")


def ldpc_profile_read(family) -> tuple[int, float]:
    fam = FAMILIES[family] if isinstance(family, str) else int(family)
    n, ms = C.c_int64(), C.c_double()
    _check(lib().ldpc_profile_read(fam, C.byref(n), C.byref(ms)), "ldpc_profile_read")
    return n.value, ms.value


def ldpc_profile_reset() -> None:
    _check(lib().ldpc_profile_reset(), "ldpc_profile_reset")


def ldpc_launch_count() -> int:
    return int(lib().ldpc_launch_count())


def ldpc_launch_count_reset() -> None:
    lib().ldpc_launch_count_reset()


# ------------------------------------------------------------------ conveniences

class Code:
    """Owns an ldpc_code handle created from a QC base matrix and lifting Z."""

    def __init__(self, base, Z: int):
        self.base = np.ascontiguousarray(base, dtype=np.int32)
        self.Z = int(Z)
        self.handle = ldpc_code_create(self.base, self.Z)
        self.N, self.K, self.M, self.E = ldpc_code_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            ldpc_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


FORMS = {
    "flood_f32": dict(sched=LDPC_SCHED_FLOODING, algo=LDPC_ALGO_SPA, msg=LDPC_MSG_F32),
    "flood_f16": dict(sched=LDPC_SCHED_FLOODING, algo=LDPC_ALGO_SPA, msg=LDPC_MSG_F16),
    "plain_f32": dict(sched=LDPC_SCHED_FLOODING, algo=LDPC_ALGO_SPA, msg=LDPC_MSG_F32, impl=LDPC_IMPL_PLAIN),
    "stream_f32": dict(sched=LDPC_SCHED_FLOODING, algo=LDPC_ALGO_SPA, msg=LDPC_MSG_F32, impl=LDPC_IMPL_STREAMING),
    "stream_f16": dict(sched=LDPC_SCHED_FLOODING, algo=LDPC_ALGO_SPA, msg=LDPC_MSG_F16, impl=LDPC_IMPL_STREAMING),
    "cluster_f32": dict(sched=LDPC_SCHED_FLOODING, algo=LDPC_ALGO_SPA, msg=LDPC_MSG_F32, impl=LDPC_IMPL_CLUSTER),
    "cluster_f16": dict(sched=LDPC_SCHED_FLOODING, algo=LDPC_ALGO_SPA, msg=LDPC_MSG_F16, impl=LDPC_IMPL_CLUSTER),
    "layered_f32": dict(sched=LDPC_SCHED_LAYERED, algo=LDPC_ALGO_SPA, msg=LDPC_MSG_F32),
    "layered_f16": dict(sched=LDPC_SCHED_LAYERED, algo=LDPC_ALGO_SPA, msg=LDPC_MSG_F16),
    "layered_i8": dict(sched=LDPC_SCHED_LAYERED, algo=LDPC_ALGO_NMS, msg=LDPC_MSG_I8),
    "layered_i8_group": dict(sched=LDPC_SCHED_LAYERED, algo=LDPC_ALGO_NMS, msg=LDPC_MSG_I8,
                             impl=LDPC_IMPL_STREAMING),
}


def params_for(form: str, **overrides) -> DecodeParams:
    kw = dict(FORMS[form])
    kw.update(overrides)
    return ldpc_default_params(**kw)


def decode(code: Code, params: DecodeParams, llr, app: bool = False, stream=None, workspace=None):
    """Decode a CUDA tensor of LLRs [n_cw, N] (fp32, or int8 for the layered form).

    Returns (bits uint8 [n_cw, N], iters int32 [n_cw], app fp32 [n_cw, N] or None) as CUDA
    tensors; the work is queued on ``stream`` (torch's current stream if None).
    """
    import torch

    if not llr.is_cuda or llr.dim() != 2 or llr.shape[1] != code.N or not llr.is_contiguous():
        raise ValueError("llr must be a contiguous CUDA tensor of shape [n_cw, N]")
    llr_type = LDPC_LLR_I8 if llr.dtype == torch.int8 else LDPC_LLR_F32
    if llr_type == LDPC_LLR_F32 and llr.dtype != torch.float32:
        raise ValueError("llr must be float32 or int8")
    n = llr.shape[0]
    bits = torch.empty((n, code.N), dtype=torch.uint8, device=llr.device)
    iters = torch.empty((n,), dtype=torch.int32, device=llr.device)
    app_t = torch.empty((n, code.N), dtype=torch.float32, device=llr.device) if app else None
    s = stream if stream is not None else torch.cuda.current_stream(llr.device)
    wsb = 0 if workspace is None else workspace.numel() * workspace.element_size()
    ldpc_decode_batch(code.handle, params, llr, llr_type, n, bits, iters, app_t, workspace, wsb, s)
    return bits, iters, app_t
