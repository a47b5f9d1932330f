"""ctypes binding of libedgb300 (include/ed.h).

Argument marshalling only: every step of the distance computation runs in the
CUDA kernels behind the C ABI.  The functions keep the C names.  Device
buffers are torch CUDA tensors (PyTorch supplies device memory and streams);
host buffers are numpy arrays, bytes, or CPU tensors (pinned or not).

There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libedgb300.so")

ED_OK, ED_EAGAIN = 0, 1
ED_EINVAL, ED_ENOMEM, ED_ECUDA, ED_ETIMEOUT, ED_EBUSY, ED_ENOTFOUND, ED_ELIMIT = -1, -2, -3, -4, -5, -6, -7
ED_LCP_AUTO, ED_LCP_DIRECT, ED_LCP_HASH, ED_LCP_BHASH = 0, 1, 2, 3
NEG32 = -1061109568  # 0xC0C0C0C0: "minus infinity" in frontier dumps


class EdError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        super().__init__(f"{what}: {_strerror(code)} ({code}){' - ' + detail if detail else ''}")


class ed_config(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int),
        ("mem_budget_bytes", ctypes.c_size_t),
        ("max_inflight", ctypes.c_int),
        ("lcp_mode", ctypes.c_int),
        ("hash_seed", ctypes.c_uint64),
        ("spin_limit_ns", ctypes.c_uint64),
        ("grid_ctas", ctypes.c_int),
        ("tile_width", ctypes.c_int),
        ("block_rounds", ctypes.c_int),
        ("max_rounds", ctypes.c_int64),
        ("hash_block", ctypes.c_int),
        ("warp_cap", ctypes.c_int),
        ("local_chunks", ctypes.c_int),
        ("help_div", ctypes.c_int),
        ("distance_hint", ctypes.c_int64),
        ("tune", ctypes.c_int),
        ("tune_table", ctypes.c_char_p),
    ]


class ed_stats(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_uint64),
        ("extensions", ctypes.c_uint64),
        ("slide_chars", ctypes.c_uint64),
        ("compared_bytes", ctypes.c_uint64),
        ("long_slides", ctypes.c_uint64),
        ("open_slides", ctypes.c_uint64),
        ("wide_rounds", ctypes.c_uint64),
        ("hash_queries", ctypes.c_uint64),
        ("hash_collisions", ctypes.c_uint64),
        ("kernel_launches", ctypes.c_uint64),
        ("kernel_ms", ctypes.c_double),
        ("build_ms", ctypes.c_double),
        ("phase_ms", ctypes.c_double * 6),
    ]


_lib = None

# name -> (restype, argtypes)
_P, _S, _I, _U64, _I64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64
_SIGS = {
    "ed_config_default": (_I, [_P]),
    "ed_tune_lookup": (_I, [ctypes.c_char_p, _S, _S, _I64, _P]),
    "ed_create": (_I, [_P, _P]),
    "ed_destroy": (_I, [_P]),
    "ed_strerror": (ctypes.c_char_p, [_I]),
    "ed_last_cuda_error": (ctypes.c_char_p, [_P]),
    "ed_distance": (_I, [_P, _P, _S, _P, _S, _P]),
    "ed_distance_dev": (_I, [_P, _P, _S, _P, _S, _P, _P]),
    "ed_last_stats": (_I, [_P, _P]),
    "ed_distance_batch_dev": (_I, [_P, _S, _P, _P, _P, _P, _P, _P]),
    "ed_distance_batch": (_I, [_P, _S, _P, _P, _P, _P, _P]),
    "ed_submit": (_I, [_P, _P, _S, _P, _S, _P]),
    "ed_submit_dev": (_I, [_P, _P, _S, _P, _S, _P, _P]),
    "ed_poll": (_I, [_P, _U64, _P]),
    "ed_serve_counters": (_I, [_P, _P, _P, _P, _P, _P]),
    "ed_lcp_dev": (_I, [_P, _P, _S, _P, _S, _P, _P, _S, _I, _P, _P, _P, _P]),
    "ed_prefix_hash_dev": (_I, [_P, _P, _S, _P, _P]),
    "ed_prefix_hash_blocked_dev": (_I, [_P, _P, _S, _S, _P, _P]),
    "ed_hash_base": (_U64, [_P]),
    "ed_frontiers_dev": (_I, [_P, _P, _S, _P, _S, _I64, _P, _P, _P]),
    "ed_edit_script_dev": (_I, [_P, _P, _S, _P, _S, _I64, _P, _S, _P, _P, _P]),
    "ed_trace_script": (_I, [_P, _I64, _S, _S, _U64, _P, _S, _P]),
    "ed_prefix_hash_noalloc": (_I, [_P, _S, _U64, _P, _P]),
}


def load(path: str = LIB_PATH):
    """Load (once) and return the library; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libedgb300 not built ({path} missing): run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _strerror(code: int) -> str:
    try:
        return load().ed_strerror(code).decode()
    except Exception:  # library missing: still format the error
        return "status"


def _check(ctx, code: int, what: str):
    if code < 0:
        detail = ""
        if ctx is not None and code in (ED_ECUDA, ED_ETIMEOUT, ED_ELIMIT):
            detail = load().ed_last_cuda_error(ctx).decode()
        raise EdError(code, what, detail)
    return code


def _host_buf(x):
    """(pointer, length, keepalive) of a host byte buffer."""
    try:
        import torch

        if isinstance(x, torch.Tensor):
            if x.is_cuda:
                raise TypeError("expected a host buffer, got a CUDA tensor")
            t = x.contiguous()
            return (t.data_ptr() if t.numel() else None), t.numel() * t.element_size(), t
    except ImportError:
        pass
    if isinstance(x, (bytes, bytearray)):
        a = np.frombuffer(bytes(x), dtype=np.uint8)
    else:
        a = np.ascontiguousarray(x, dtype=np.uint8)
    return (a.ctypes.data if a.size else None), a.size, a


def _dev_buf(t):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != torch.uint8:
        raise TypeError("expected a uint8 tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return (t.data_ptr() if t.numel() else None), t.numel()


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- the ABI
def ed_config_default() -> ed_config:
    c = ed_config()
    _check(None, load().ed_config_default(ctypes.byref(c)), "ed_config_default")
    return c


def ed_tune_lookup(n: int, m: int, distance_hint: int = 0, table: str | None = None) -> ed_config:
    """The tuning-table row for lengths n, m (include/ed.h), as an ed_config
    whose other fields are the defaults."""
    c = ed_config_default()
    _check(None, load().ed_tune_lookup(table.encode() if table else None, n, m, distance_hint, ctypes.byref(c)),
           "ed_tune_lookup")
    return c


def ed_create(cfg: ed_config | None = None):
    h = ctypes.c_void_p()
    _check(None, load().ed_create(ctypes.byref(h), ctypes.byref(cfg) if cfg is not None else None),
           "ed_create")
    return h


def ed_destroy(ctx) -> None:
    _check(None, load().ed_destroy(ctx), "ed_destroy")


def ed_strerror(code: int) -> str:
    return load().ed_strerror(code).decode()


def ed_distance(ctx, A, B) -> int:
    pa, n, ka = _host_buf(A)
    pb, m, kb = _host_buf(B)
    k = ctypes.c_uint64()
    _check(ctx, load().ed_distance(ctx, pa, n, pb, m, ctypes.byref(k)), "ed_distance")
    return int(k.value)


def ed_distance_dev(ctx, A, B, stream=None) -> int:
    pa, n = _dev_buf(A)
    pb, m = _dev_buf(B)
    k = ctypes.c_uint64()
    _check(ctx, load().ed_distance_dev(ctx, pa, n, pb, m, ctypes.byref(k), _stream_ptr(stream)),
           "ed_distance_dev")
    return int(k.value)


def ed_last_stats(ctx) -> dict:
    s = ed_stats()
    _check(ctx, load().ed_last_stats(ctx, ctypes.byref(s)), "ed_last_stats")
    d = {f: getattr(s, f) for f, _ in ed_stats._fields_}
    d["phase_ms"] = list(d["phase_ms"])
    return d


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * max(1, len(ptrs)))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


def ed_distance_batch_dev(ctx, As: Sequence, Bs: Sequence, stream=None) -> np.ndarray:
    npairs = len(As)
    pa = [_dev_buf(a) for a in As]
    pb = [_dev_buf(b) for b in Bs]
    n = np.array([x[1] for x in pa], dtype=np.uint64)
    m = np.array([x[1] for x in pb], dtype=np.uint64)
    out = np.zeros(max(1, npairs), dtype=np.uint64)
    _check(ctx, load().ed_distance_batch_dev(
        ctx, npairs, _ptr_array([x[0] for x in pa]), n.ctypes.data if npairs else None,
        _ptr_array([x[0] for x in pb]), m.ctypes.data if npairs else None,
        out.ctypes.data, _stream_ptr(stream)), "ed_distance_batch_dev")
    return out[:npairs].astype(np.int64)


def ed_distance_batch(ctx, As: Sequence, Bs: Sequence) -> np.ndarray:
    npairs = len(As)
    ha = [_host_buf(a) for a in As]
    hb = [_host_buf(b) for b in Bs]
    n = np.array([x[1] for x in ha], dtype=np.uint64)
    m = np.array([x[1] for x in hb], dtype=np.uint64)
    out = np.zeros(max(1, npairs), dtype=np.uint64)
    _check(ctx, load().ed_distance_batch(
        ctx, npairs, _ptr_array([x[0] for x in ha]), n.ctypes.data if npairs else None,
        _ptr_array([x[0] for x in hb]), m.ctypes.data if npairs else None, out.ctypes.data),
        "ed_distance_batch")
    return out[:npairs].astype(np.int64)


def ed_submit(ctx, A, B) -> int:
    """Returns a ticket, or raises EdError(ED_EBUSY) when not admitted."""
    pa, n, ka = _host_buf(A)
    pb, m, kb = _host_buf(B)
    t = ctypes.c_uint64()
    _check(ctx, load().ed_submit(ctx, pa, n, pb, m, ctypes.byref(t)), "ed_submit")
    return int(t.value)


def ed_submit_dev(ctx, A, B, stream=None) -> int:
    """Submits device strings (CUDA uint8 tensors) written on `stream`;
    they must stay alive until the ticket is polled done."""
    pa, n = _dev_buf(A)
    pb, m = _dev_buf(B)
    t = ctypes.c_uint64()
    _check(ctx, load().ed_submit_dev(ctx, pa, n, pb, m, ctypes.byref(t), _stream_ptr(stream)), "ed_submit_dev")
    return int(t.value)


def ed_poll(ctx, ticket: int):
    """(status, k): status ED_OK with k, or ED_EAGAIN; errors raise."""
    k = ctypes.c_uint64()
    r = load().ed_poll(ctx, ticket, ctypes.byref(k))
    if r == ED_EAGAIN:
        return ED_EAGAIN, None
    _check(ctx, r, "ed_poll")
    return ED_OK, int(k.value)


def ed_serve_counters(ctx) -> dict:
    v = [ctypes.c_uint64() for _ in range(5)]
    _check(ctx, load().ed_serve_counters(ctx, *[ctypes.byref(x) for x in v]), "ed_serve_counters")
    return dict(zip(["admitted", "completed", "inflight", "steps", "slices"], [int(x.value) for x in v]))


def ed_lcp_dev(ctx, A, B, x, y, method: int, TA=None, TB=None, stream=None) -> np.ndarray:
    pa, n = _dev_buf(A)
    pb, m = _dev_buf(B)
    xs = np.ascontiguousarray(x, dtype=np.int64)
    ys = np.ascontiguousarray(y, dtype=np.int64)
    out = np.zeros(max(1, xs.size), dtype=np.int64)
    ta = TA.data_ptr() if TA is not None else None
    tb = TB.data_ptr() if TB is not None else None
    _check(ctx, load().ed_lcp_dev(ctx, pa, n, pb, m, xs.ctypes.data, ys.ctypes.data, xs.size, method,
                                  ta, tb, out.ctypes.data, _stream_ptr(stream)), "ed_lcp_dev")
    return out[: xs.size]


def ed_prefix_hash_dev(ctx, X, stream=None):
    """T[0..len] as an int64 CUDA tensor holding the uint64 hash values."""
    import torch

    px, n = _dev_buf(X)
    T = torch.empty(n + 1, dtype=torch.int64, device=X.device)
    _check(ctx, load().ed_prefix_hash_dev(ctx, px, n, T.data_ptr(), _stream_ptr(stream)),
           "ed_prefix_hash_dev")
    return T


def ed_prefix_hash_blocked_dev(ctx, X, b: int, stream=None):
    """T[0..len//b] (block prefixes of Sec. 3.3) as an int64 CUDA tensor."""
    import torch

    px, n = _dev_buf(X)
    T = torch.empty(n // b + 1, dtype=torch.int64, device=X.device)
    _check(ctx, load().ed_prefix_hash_blocked_dev(ctx, px, n, b, T.data_ptr(), _stream_ptr(stream)),
           "ed_prefix_hash_blocked_dev")
    return T


def ed_hash_base(ctx) -> int:
    return int(load().ed_hash_base(ctx))


ED_NOALLOC_MAX_LEN = 89468928


def ed_prefix_hash_noalloc(X, base: int, T, stream=None) -> None:
    """The prefix table of X into the caller's CUDA tensor T (int64, len+1
    entries) without any allocation by the library (include/ed.h).  X, T
    and the stream must be on one device; the call runs with that device
    current."""
    import torch

    px, n = _dev_buf(X)
    if not isinstance(T, torch.Tensor) or not T.is_cuda or T.element_size() != 8 or T.numel() != n + 1:
        raise ValueError("T must be a CUDA tensor of len(X) + 1 8-byte entries")
    if not T.is_contiguous():
        raise ValueError("T must be contiguous")
    if T.device != X.device:
        raise ValueError("X and T must be on the same device")
    with torch.cuda.device(X.device):
        if stream is None:
            stream = torch.cuda.current_stream(X.device)
        elif stream.device != X.device:
            raise ValueError("the stream must belong to the device of X and T")
        _check(None, load().ed_prefix_hash_noalloc(px, n, base, T.data_ptr(), _stream_ptr(stream)),
               "ed_prefix_hash_noalloc")


def ed_frontiers_dev(ctx, A, B, t_max: int, stream=None):
    """(k or None if k > t_max, F) with F[t, d + t_max] = L_t[d] (NEG32 where undefined)."""
    pa, n = _dev_buf(A)
    pb, m = _dev_buf(B)
    F = np.empty((t_max + 1, 2 * t_max + 1), dtype=np.int32)
    k = ctypes.c_uint64()
    _check(ctx, load().ed_frontiers_dev(ctx, pa, n, pb, m, t_max, F.ctypes.data, ctypes.byref(k),
                                        _stream_ptr(stream)), "ed_frontiers_dev")
    kk = int(k.value)
    return (None if kk == 2**64 - 1 else kk), F


ED_OP_SUB, ED_OP_DEL, ED_OP_INS = 0, 1, 2


def ed_edit_script_dev(ctx, A, B, t_max: int, stream=None):
    """(k, ops) with ops an (k, 3) int64 array of (kind, x, y): an optimal
    edit script of A into B, in order from the start of the strings."""
    pa, n = _dev_buf(A)
    pb, m = _dev_buf(B)
    ops = np.zeros((max(t_max, 1), 3), dtype=np.int64)
    nops = ctypes.c_size_t()
    k = ctypes.c_uint64()
    _check(ctx, load().ed_edit_script_dev(ctx, pa, n, pb, m, t_max, ops.ctypes.data, t_max, ctypes.byref(nops),
                                          ctypes.byref(k), _stream_ptr(stream)), "ed_edit_script_dev")
    return int(k.value), ops[: int(nops.value)].copy()


def ed_trace_script(F, t_max: int, n: int, m: int, k: int):
    """ops (k, 3) int64 traced back from host frontiers F[t, d + t_max] = L_t[d]."""
    F = np.ascontiguousarray(F, dtype=np.int32)
    assert F.shape[1] == 2 * t_max + 1 and F.shape[0] >= k + 1
    ops = np.zeros((max(k, 1), 3), dtype=np.int64)
    nops = ctypes.c_size_t()
    _check(None, load().ed_trace_script(F.ctypes.data, t_max, n, m, k, ops.ctypes.data, k, ctypes.byref(nops)),
           "ed_trace_script")
    return ops[: int(nops.value)].copy()


class Context:
    """Owns one ed_ctx; a thin convenience over the functions above."""

    def __init__(self, **cfg):
        c = ed_config_default()
        for key, v in cfg.items():
            if key == "tune_table" and isinstance(v, str):
                v = v.encode()
            setattr(c, key, v)
        self.cfg = c
        self.h = ed_create(c)

    def close(self):
        if self.h:
            ed_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def distance(self, A, B) -> int:
        return ed_distance(self.h, A, B)

    def distance_dev(self, A, B, stream=None) -> int:
        return ed_distance_dev(self.h, A, B, stream)

    def stats(self) -> dict:
        return ed_last_stats(self.h)
