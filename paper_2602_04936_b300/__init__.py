"""Python binding of liblcp.so -- deterministic top-k LCP retrieval on B300.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of liblcp.so (C ABI declared in include/lcp.h).  PyTorch supplies
device memory and the current CUDA stream.  There is no CPU fallback: if the
shared library cannot be loaded, importing this package raises.

Names mirror the C entry points:

    idx = lcp_index_build(tokens, max_k=128, capacity=0)     # Algorithm 1
    lcp_index_insert(idx, new_tokens)                        # ids N, N+1, ...
    ids, lcp = lcp_topk_batch(idx, queries, k)               # Algorithms 3/4
    ids, lcp = lcp_scan_topk(tokens, queries, k)             # full scan
    ids, lcp = lcp_topk_batch_host(idx, host_queries, k)     # host buffers

Tokens are [n, L] tensors of 1-byte (uint8) or 2-byte (uint16 / int16,
reinterpreted as unsigned) elements.  Results are ([Q, k] int32 ids,
[Q, k] uint8 LCPs), ordered by (LCP desc, id asc), padded with (-1, 0).
"""
from __future__ import annotations

import ctypes
import os
import sys

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liblcp.so")

LCP_OK = 0
LCP_PENDING = 1
LCP_ERR_INVALID = -1
LCP_ERR_OOM = -2
LCP_ERR_CAPACITY = -3
LCP_ERR_BUDGET = -4
LCP_ERR_TIMEOUT = -5
LCP_ERR_CUDA = -6
LCP_ERR_STATE = -7
LCP_INDEX_MAX_K = 128
LCP_SCAN_MAX_K = 1024
LCP_INSERT_SMALL_BATCH = 2048
LCP_MAX_L = 255
LCP_MAX_L_WIDE = 1024

# Every symbol include/lcp.h declares (checked by the CPU test suite).
ABI_SYMBOLS = (
    "lcp_status_string", "lcp_index_build", "lcp_index_build_host", "lcp_index_insert",
    "lcp_topk_batch", "lcp_topk_batch_host", "lcp_scan_topk", "lcp_index_size",
    "lcp_index_export", "lcp_index_sync", "lcp_index_destroy", "lcp_device_status",
    "lcp_launch_count", "lcp_debug_bounded_wait", "lcp_scan_topk_noalloc",
    "lcp_kernel_timing", "lcp_kernel_time", "lcp_kernel_timing_filter", "lcp_build_graph",
    "lcp_session_create", "lcp_session_add_index", "lcp_session_add_scan", "lcp_session_submit",
    "lcp_session_poll",
    "lcp_session_stats", "lcp_session_destroy", "lcp_session_replay",
    "lcp_step_create", "lcp_step_run", "lcp_step_stats", "lcp_step_destroy", "lcp_shard_merge",
    "lcp_topk_bfs", "lcp_tal_topk",
    "lcp_queue_create", "lcp_queue_submit", "lcp_queue_poll", "lcp_queue_stats", "lcp_queue_destroy",
    "lcp_queue_replay", "lcp_autotune", "lcp_set_search_shape", "lcp_top1_wide", "lcp_scan_top1_wide",
)


class LcpError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, _lib.lcp_status_string(code).decode(), code))


class _Format(ctypes.Structure):
    _fields_ = [("token_bytes", ctypes.c_int32), ("L", ctypes.c_int32), ("vocab", ctypes.c_int32)]


class SessionConfig(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("dry_run", ctypes.c_int32)]


class ReplayRequest(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("slot", ctypes.c_int32), ("k", ctypes.c_int32),
                ("Q", ctypes.c_int64), ("h_queries", ctypes.c_void_p), ("h_out_ids", ctypes.c_void_p),
                ("h_out_lcp", ctypes.c_void_p)]


class QueueConfig(ctypes.Structure):
    _fields_ = [("max_requests", ctypes.c_int32), ("max_tasks", ctypes.c_int32), ("idle_ms", ctypes.c_double),
                ("ctas_per_sm", ctypes.c_int32)]


class QueueReplayRequest(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("index", ctypes.c_void_p), ("k", ctypes.c_int32),
                ("Q", ctypes.c_int64), ("d_queries", ctypes.c_void_p), ("d_out_ids", ctypes.c_void_p),
                ("d_out_lcp", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("qpw", ctypes.c_int32), ("locate_warp", ctypes.c_int32), ("best_ms", ctypes.c_float),
                ("default_ms", ctypes.c_float)]


class SessionStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "admitted", "completed", "rejected",
                                                "inflight", "pending", "mem_in_use", "mem_peak")]


def _load():
    try:  # (re)build when a source is newer than liblcp.so; a no-op otherwise
        from . import build as _b
        _b.build()
    except Exception as e:
        if not os.path.exists(_SO):  # no CPU fallback: fail loudly
            raise ImportError("liblcp.so is missing and could not be built: %s" % e) from e
    lib = ctypes.CDLL(_SO)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    sig = {
        "lcp_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "lcp_index_build": ([vp, i64, _Format, i64, i32, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "lcp_index_build_host": ([vp, i64, _Format, i64, i32, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "lcp_index_insert": ([vp, vp, i64, vp], ctypes.c_int),
        "lcp_topk_batch": ([vp, vp, i64, i32, vp, vp, vp], ctypes.c_int),
        "lcp_topk_batch_host": ([vp, vp, i64, i32, vp, vp, vp], ctypes.c_int),
        "lcp_scan_topk": ([vp, i64, _Format, vp, i64, i32, vp, vp, vp], ctypes.c_int),
        "lcp_index_size": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "lcp_index_export": ([vp, vp, vp, vp], ctypes.c_int),
        "lcp_index_sync": ([vp], ctypes.c_int),
        "lcp_index_destroy": ([vp], ctypes.c_int),
        "lcp_device_status": ([], ctypes.c_int),
        "lcp_launch_count": ([], i64),
        "lcp_kernel_timing": ([ctypes.c_int], ctypes.c_int),
        "lcp_build_graph": ([ctypes.c_int], ctypes.c_int),
        "lcp_kernel_timing_filter": ([ctypes.c_char_p], ctypes.c_int),
        "lcp_kernel_time": ([ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)],
                            ctypes.c_int),
        "lcp_debug_bounded_wait": ([i64, vp], ctypes.c_int),
        "lcp_scan_topk_noalloc": ([vp, i64, _Format, vp, i64, i32, vp, vp, vp], ctypes.c_int),
        "lcp_top1_wide": ([vp, vp, i64, vp, vp, vp], ctypes.c_int),
        "lcp_scan_top1_wide": ([vp, i64, _Format, vp, i64, vp, vp, vp], ctypes.c_int),
        "lcp_session_create": ([ctypes.POINTER(SessionConfig), ctypes.POINTER(vp)], ctypes.c_int),
        "lcp_session_add_index": ([vp, vp, ctypes.POINTER(i32)], ctypes.c_int),
        "lcp_session_add_scan": ([vp, vp, i64, _Format, ctypes.POINTER(i32)], ctypes.c_int),
        "lcp_session_submit": ([vp, i32, vp, i64, i32, vp, vp, ctypes.POINTER(ctypes.c_uint64)],
                               ctypes.c_int),
        "lcp_session_poll": ([vp, ctypes.c_uint64, i32], ctypes.c_int),
        "lcp_session_stats": ([vp, ctypes.POINTER(SessionStats)], ctypes.c_int),
        "lcp_session_destroy": ([vp], ctypes.c_int),
        "lcp_session_replay": ([vp, ctypes.POINTER(ReplayRequest), i64, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                               ctypes.c_int),
        "lcp_step_create": ([vp, i64, i64, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "lcp_step_run": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "lcp_step_stats": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "lcp_step_destroy": ([vp], ctypes.c_int),
        "lcp_shard_merge": ([vp, vp, i32, ctypes.POINTER(i64), i64, i32, vp, vp, vp], ctypes.c_int),
        "lcp_topk_bfs": ([vp, vp, i64, i32, vp, vp, vp], ctypes.c_int),
        "lcp_tal_topk": ([vp, vp, i64, i32, i32, vp, vp, vp], ctypes.c_int),
        "lcp_queue_create": ([ctypes.POINTER(QueueConfig), ctypes.POINTER(vp)], ctypes.c_int),
        "lcp_queue_submit": ([vp, vp, vp, i64, i32, vp, vp, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "lcp_queue_poll": ([vp, ctypes.c_uint64, i32], ctypes.c_int),
        "lcp_queue_stats": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "lcp_queue_destroy": ([vp], ctypes.c_int),
        "lcp_autotune": ([vp, vp, i64, i32, vp, ctypes.POINTER(TuneResult)], ctypes.c_int),
        "lcp_set_search_shape": ([vp, i64, i32, i32, i32], ctypes.c_int),
        "lcp_queue_replay": ([vp, ctypes.POINTER(QueueReplayRequest), i64, ctypes.c_double,
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def library_path() -> str:
    return _SO


def _check(rc: int, what: str):
    if rc != LCP_OK:
        raise LcpError(rc, what)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _token_bytes(t: torch.Tensor) -> int:
    es = t.element_size()
    if es not in (1, 2) or t.is_floating_point():
        raise TypeError("tokens must be 1- or 2-byte integers, got %s" % t.dtype)
    return es


def _rows(t: torch.Tensor, device: bool):
    if t.dim() != 2:
        raise ValueError("tokens must be [n, L]")
    if device and not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not device and t.is_cuda:
        raise ValueError("expected a host tensor")
    return t.contiguous()


def _fmt(t: torch.Tensor, vocab: int = 0) -> _Format:
    return _Format(_token_bytes(t), t.shape[1], vocab)


class _NoSwitch:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


_NO_SWITCH = _NoSwitch()


def _on(device):
    """The device's context, entered only when it is not already current
    (a device switch costs a few microseconds a call)."""
    idx = device.index if isinstance(device, torch.device) else device
    if idx is None or idx == torch.cuda.current_device():
        return _NO_SWITCH
    return torch.cuda.device(device)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else ctypes.c_void_p(0)


class Index:
    """Owning handle of a device-resident prefix index."""

    def __init__(self, handle: ctypes.c_void_p, L: int, token_bytes: int, max_k: int, device):
        self._h = handle
        self.L, self.token_bytes, self.max_k, self.device = L, token_bytes, max_k, device

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise LcpError(LCP_ERR_STATE, "index")
        return self._h

    def size(self):
        n, b = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.lcp_index_size(self.handle, ctypes.byref(n), ctypes.byref(b)), "lcp_index_size")
        return n.value, b.value

    @property
    def N(self) -> int:
        return self.size()[0]

    def close(self):
        if self._h is not None and self._h.value:
            _lib.lcp_index_destroy(self._h)
        self._h = None

    def __del__(self):
        if sys.is_finalizing():  # CUDA may already be torn down: leak, do not call in
            return
        try:
            self.close()
        except Exception:
            pass


def lcp_status_string(code: int) -> str:
    return _lib.lcp_status_string(code).decode()


def lcp_index_build(tokens: torch.Tensor, max_k: int = LCP_INDEX_MAX_K, capacity: int = 0,
                    vocab: int = 0, stream=None) -> Index:
    tokens = _rows(tokens, device=True)
    h = ctypes.c_void_p()
    with _on(tokens.device):
        rc = _lib.lcp_index_build(_ptr(tokens), tokens.shape[0], _fmt(tokens, vocab), capacity, max_k,
                                  _stream(stream), ctypes.byref(h))
    _check(rc, "lcp_index_build")
    return Index(h, tokens.shape[1], _token_bytes(tokens), max_k, tokens.device)


def lcp_index_build_host(tokens: torch.Tensor, max_k: int = LCP_INDEX_MAX_K, capacity: int = 0,
                         vocab: int = 0, stream=None, device=None) -> Index:
    tokens = _rows(tokens, device=False)
    h = ctypes.c_void_p()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with _on(dev):
        rc = _lib.lcp_index_build_host(_ptr(tokens), tokens.shape[0], _fmt(tokens, vocab), capacity,
                                       max_k, _stream(stream), ctypes.byref(h))
    _check(rc, "lcp_index_build_host")
    return Index(h, tokens.shape[1], _token_bytes(tokens), max_k, dev)


def lcp_index_insert(index: Index, tokens: torch.Tensor, stream=None) -> None:
    tokens = _rows(tokens, device=True)
    if tokens.shape[1] != index.L or _token_bytes(tokens) != index.token_bytes:
        raise ValueError("insert batch format differs from the index")
    with _on(tokens.device):
        _check(_lib.lcp_index_insert(index.handle, _ptr(tokens), tokens.shape[0], _stream(stream)),
               "lcp_index_insert")


def _outputs(Q, k, device, out_ids, out_lcp, pin=False):
    if out_ids is None:
        out_ids = torch.empty((Q, k), dtype=torch.int32, device=device, pin_memory=pin)
    if out_lcp is None:
        out_lcp = torch.empty((Q, k), dtype=torch.uint8, device=device, pin_memory=pin)
    if out_ids.dtype != torch.int32 or out_lcp.dtype != torch.uint8:
        raise TypeError("outputs must be int32 ids and uint8 LCPs")
    if tuple(out_ids.shape) != (Q, k) or tuple(out_lcp.shape) != (Q, k):
        raise ValueError("outputs must be [Q, k]")
    if not (out_ids.is_contiguous() and out_lcp.is_contiguous()):
        raise ValueError("outputs must be contiguous")
    return out_ids, out_lcp


def lcp_topk_batch(index: Index, queries: torch.Tensor, k: int, out_ids=None, out_lcp=None,
                   stream=None):
    queries = _rows(queries, device=True)
    if queries.shape[1] != index.L or _token_bytes(queries) != index.token_bytes:
        raise ValueError("query format differs from the index")
    Q = queries.shape[0]
    out_ids, out_lcp = _outputs(Q, k, queries.device, out_ids, out_lcp)
    with _on(queries.device):
        _check(_lib.lcp_topk_batch(index.handle, _ptr(queries), Q, k, _ptr(out_ids), _ptr(out_lcp),
                                   _stream(stream)), "lcp_topk_batch")
    return out_ids, out_lcp


def lcp_topk_batch_host(index: Index, queries: torch.Tensor, k: int, out_ids=None, out_lcp=None,
                        stream=None):
    queries = _rows(queries, device=False)
    Q = queries.shape[0]
    out_ids, out_lcp = _outputs(Q, k, "cpu", out_ids, out_lcp, pin=False)
    with _on(index.device):
        _check(_lib.lcp_topk_batch_host(index.handle, _ptr(queries), Q, k, _ptr(out_ids),
                                        _ptr(out_lcp), _stream(stream)), "lcp_topk_batch_host")
    return out_ids, out_lcp


def lcp_scan_topk(tokens: torch.Tensor, queries: torch.Tensor, k: int, out_ids=None, out_lcp=None,
                  stream=None, vocab: int = 0):
    tokens = _rows(tokens, device=True)
    queries = _rows(queries, device=True)
    if queries.shape[1] != tokens.shape[1] or _token_bytes(queries) != _token_bytes(tokens):
        raise ValueError("query format differs from the tokens")
    Q = queries.shape[0]
    out_ids, out_lcp = _outputs(Q, k, queries.device, out_ids, out_lcp)
    with _on(queries.device):
        _check(_lib.lcp_scan_topk(_ptr(tokens), tokens.shape[0], _fmt(tokens, vocab), _ptr(queries), Q,
                                  k, _ptr(out_ids), _ptr(out_lcp), _stream(stream)), "lcp_scan_topk")
    return out_ids, out_lcp


def lcp_scan_topk_noalloc(tokens: torch.Tensor, queries: torch.Tensor, k: int, out_ids, out_lcp,
                          stream=None, vocab: int = 0):
    """Full scan into caller-provided outputs, using only the library's fixed
    device scratch (no allocation in the library call; see include/lcp.h)."""
    tokens = _rows(tokens, device=True)
    queries = _rows(queries, device=True)
    Q = queries.shape[0]
    out_ids, out_lcp = _outputs(Q, k, queries.device, out_ids, out_lcp)
    with _on(queries.device):
        _check(_lib.lcp_scan_topk_noalloc(_ptr(tokens), tokens.shape[0], _fmt(tokens, vocab),
                                          _ptr(queries), Q, k, _ptr(out_ids), _ptr(out_lcp),
                                          _stream(stream)), "lcp_scan_topk_noalloc")
    return out_ids, out_lcp


def _outputs_wide(Q, device, out_ids, out_lcp):
    if out_ids is None:
        out_ids = torch.empty(Q, dtype=torch.int32, device=device)
    if out_lcp is None:
        out_lcp = torch.empty(Q, dtype=torch.int16, device=device)  # uint16 values, viewed signed
    if out_ids.dtype != torch.int32 or out_lcp.element_size() != 2 or out_lcp.is_floating_point():
        raise TypeError("outputs must be int32 ids and 16-bit LCPs")
    if out_ids.numel() != Q or out_lcp.numel() != Q or not (out_ids.is_contiguous() and out_lcp.is_contiguous()):
        raise ValueError("outputs must be contiguous [Q]")
    return out_ids, out_lcp


def lcp_top1_wide(index: Index, queries: torch.Tensor, out_ids=None, out_lcp=None, stream=None):
    """Top-1 with 16-bit LCPs (rows of up to LCP_MAX_L_WIDE tokens): (ids [Q]
    int32, lcp [Q] int16 holding the uint16 values)."""
    queries = _rows(queries, device=True)
    if queries.shape[1] != index.L or _token_bytes(queries) != index.token_bytes:
        raise ValueError("query format differs from the index")
    Q = queries.shape[0]
    out_ids, out_lcp = _outputs_wide(Q, queries.device, out_ids, out_lcp)
    with _on(queries.device):
        _check(_lib.lcp_top1_wide(index.handle, _ptr(queries), Q, _ptr(out_ids), _ptr(out_lcp), _stream(stream)),
               "lcp_top1_wide")
    return out_ids, out_lcp


def lcp_scan_top1_wide(tokens: torch.Tensor, queries: torch.Tensor, out_ids=None, out_lcp=None, stream=None,
                       vocab: int = 0):
    """Full-scan top-1 with 16-bit LCPs: (ids [Q] int32, lcp [Q] int16
    holding the uint16 values)."""
    tokens = _rows(tokens, device=True)
    queries = _rows(queries, device=True)
    if queries.shape[1] != tokens.shape[1] or _token_bytes(queries) != _token_bytes(tokens):
        raise ValueError("query format differs from the tokens")
    Q = queries.shape[0]
    out_ids, out_lcp = _outputs_wide(Q, queries.device, out_ids, out_lcp)
    with _on(queries.device):
        _check(_lib.lcp_scan_top1_wide(_ptr(tokens), tokens.shape[0], _fmt(tokens, vocab), _ptr(queries), Q,
                                       _ptr(out_ids), _ptr(out_lcp), _stream(stream)), "lcp_scan_top1_wide")
    return out_ids, out_lcp


def lcp_index_export(index: Index, stream=None):
    """(ids [N] int32, H [N] uint8) of the sorted index, on the index's device
    (H is None for an index of rows longer than LCP_MAX_L tokens)."""
    n = index.N
    ids = torch.empty(n, dtype=torch.int32, device=index.device)
    H = torch.empty(n, dtype=torch.uint8, device=index.device) if index.L <= LCP_MAX_L else None
    with _on(index.device):
        _check(_lib.lcp_index_export(index.handle, _ptr(ids), _ptr(H), _stream(stream)),
               "lcp_index_export")
    return ids, H


def lcp_index_sync(index: Index) -> int:
    return _lib.lcp_index_sync(index.handle)


def lcp_index_size(index: Index):
    return index.size()


def lcp_index_destroy(index: Index) -> None:
    index.close()


def lcp_device_status() -> int:
    return _lib.lcp_device_status()


def lcp_launch_count() -> int:
    return int(_lib.lcp_launch_count())


def lcp_kernel_timing(enable: bool) -> None:
    """Per-kernel CUDA-event timing on/off (enabling clears the totals)."""
    _check(_lib.lcp_kernel_timing(1 if enable else 0), "lcp_kernel_timing")


def lcp_build_graph(enable: bool) -> None:
    """Builds as one replayed CUDA graph (the default) or by direct launches,
    which per-kernel timing can bracket."""
    _check(_lib.lcp_build_graph(1 if enable else 0), "lcp_build_graph")


def lcp_kernel_timing_filter(prefix: str = "") -> None:
    """Time only kernels whose name starts with prefix ("" = all)."""
    _check(_lib.lcp_kernel_timing_filter(prefix.encode()), "lcp_kernel_timing_filter")


def lcp_kernel_time(prefix: str):
    """(total device ms, launches) of timed kernels whose name starts with prefix."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(_lib.lcp_kernel_time(prefix.encode(), ctypes.byref(ms), ctypes.byref(n)), "lcp_kernel_time")
    return ms.value, n.value


def lcp_debug_bounded_wait(spin_limit: int, stream=None) -> int:
    return _lib.lcp_debug_bounded_wait(spin_limit, _stream(stream))


LCP_SHARD_MAX = 32
LCP_TAL_MAX_K = 32


def lcp_autotune(index: "Index", queries: torch.Tensor, k: int, stream=None) -> dict:
    """Times every search launch shape on this sample batch and installs the
    fastest for batches of the same class (see lcp.h)."""
    q = _rows(queries, True)
    r = TuneResult()
    with _on(q.device):
        _check(_lib.lcp_autotune(index.handle, _ptr(q), q.shape[0], k, _stream(stream), ctypes.byref(r)),
               "lcp_autotune")
    return {"qpw": r.qpw, "locate_warp": r.locate_warp, "best_ms": r.best_ms, "default_ms": r.default_ms}


def lcp_set_search_shape(index: "Index", Q: int, k: int, qpw: int, locate_warp: int) -> None:
    _check(_lib.lcp_set_search_shape(index.handle, Q, k, qpw, locate_warp), "lcp_set_search_shape")


def lcp_topk_bfs(index: "Index", queries: torch.Tensor, k: int, out_ids=None, out_lcp=None, stream=None):
    """Algorithms 3 + 4 as printed: first k items of the deepest node's subtree
    in BFS (sorted-row) order, each with the descent depth as LCP."""
    q = _rows(queries, True)
    if q.shape[1] != index.L or _token_bytes(q) != index.token_bytes:
        raise ValueError("query format differs from the index")
    out_ids, out_lcp = _outputs(q.shape[0], k, q.device, out_ids, out_lcp)
    with _on(q.device):
        _check(_lib.lcp_topk_bfs(index.handle, _ptr(q), q.shape[0], k, _ptr(out_ids), _ptr(out_lcp),
                                 _stream(stream)), "lcp_topk_bfs")
    return out_ids, out_lcp


def lcp_tal_topk(index: "Index", queries: torch.Tensor, k: int, depth: int, out_ids=None, out_lcp=None,
                 stream=None):
    """TAL bucket scan: top k of the rows sharing each query's first `depth`
    tokens, found by scanning that bucket only."""
    q = _rows(queries, True)
    if q.shape[1] != index.L or _token_bytes(q) != index.token_bytes:
        raise ValueError("query format differs from the index")
    out_ids, out_lcp = _outputs(q.shape[0], k, q.device, out_ids, out_lcp)
    with _on(q.device):
        _check(_lib.lcp_tal_topk(index.handle, _ptr(q), q.shape[0], k, depth, _ptr(out_ids), _ptr(out_lcp),
                                 _stream(stream)), "lcp_tal_topk")
    return out_ids, out_lcp


def lcp_shard_merge(ids: torch.Tensor, lcp: torch.Tensor, bases, out_ids=None, out_lcp=None, stream=None):
    """Global top k from P shard answers: ids/lcp [P, Q, k] (device, each
    shard's lcp_topk_batch output with local ids), bases = first global id of
    each shard.  Returns ([Q, k] int32, [Q, k] uint8)."""
    if ids.dim() != 3 or tuple(lcp.shape) != tuple(ids.shape):
        raise ValueError("ids and lcp must both be [P, Q, k]")
    if ids.dtype != torch.int32 or lcp.dtype != torch.uint8:
        raise TypeError("ids must be int32 and lcp uint8")
    P, Q, k = ids.shape
    if len(bases) != P:
        raise ValueError("one base per shard")
    hb = (ctypes.c_int64 * P)(*[int(b) for b in bases])
    out_ids, out_lcp = _outputs(Q, k, ids.device, out_ids, out_lcp)
    with _on(ids.device):
        _check(_lib.lcp_shard_merge(_ptr(ids.contiguous()), _ptr(lcp.contiguous()), P, hb, Q, k,
                                    _ptr(out_ids), _ptr(out_lcp), _stream(stream)), "lcp_shard_merge")
    return out_ids, out_lcp


class Queue:
    """Persistent search kernel fed by a work queue (lcp.h): submit requests
    against any resident index, poll their tickets."""

    def __init__(self, max_requests: int = 256, max_tasks: int = 1 << 16, idle_ms: float = 2.0,
                 ctas_per_sm: int = 4):
        self._h = ctypes.c_void_p()
        cfg = QueueConfig(max_requests, max_tasks, idle_ms, ctas_per_sm)
        _check(_lib.lcp_queue_create(ctypes.byref(cfg), ctypes.byref(self._h)), "lcp_queue_create")
        self._live = {}  # ticket -> tensors that must outlive the request

    def submit(self, index: "Index", queries: torch.Tensor, k: int, out_ids=None, out_lcp=None) -> int:
        """Queries must be device-resident and fully written (stream synchronized)."""
        q = _rows(queries, True)
        if q.shape[1] != index.L or _token_bytes(q) != index.token_bytes:
            raise ValueError("query format differs from the index")
        out_ids, out_lcp = _outputs(q.shape[0], k, q.device, out_ids, out_lcp)
        t = ctypes.c_uint64()
        _check(_lib.lcp_queue_submit(self._h, index.handle, _ptr(q), q.shape[0], k, _ptr(out_ids), _ptr(out_lcp),
                                     ctypes.byref(t)), "lcp_queue_submit")
        self._live[t.value] = (index, q, out_ids, out_lcp)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0) -> int:
        """LCP_OK once complete, LCP_PENDING at the timeout."""
        return _lib.lcp_queue_poll(self._h, ticket, timeout_ms)

    def result(self, ticket: int, timeout_ms: int = 10_000):
        """Waits for the request and hands back its (ids, lcp) outputs."""
        _check(self.poll(ticket, timeout_ms), "lcp_queue_poll")
        held = self._live.pop(ticket)
        return held[2], held[3]

    def replay(self, reqs, timeout_s: float = 60.0):
        """Native open-loop replay of QueueReplayRequest records: (rc,
        latencies in seconds, wall seconds)."""
        import numpy as np
        n = len(reqs)
        arr = (QueueReplayRequest * n)(*reqs)
        lat = np.zeros(n, np.float64)
        wall = ctypes.c_double()
        rc = _lib.lcp_queue_replay(self._h, arr, n, timeout_s, lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(wall))
        return rc, lat, wall.value

    def stats(self):
        n, l = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.lcp_queue_stats(self._h, ctypes.byref(n), ctypes.byref(l)), "lcp_queue_stats")
        return {"inflight": n.value, "worker_launches": l.value}

    def close(self):
        if self._h is not None and self._h.value:
            _lib.lcp_queue_destroy(self._h)
            self._live.clear()
        self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Step:
    """Insert-then-query streaming step replayed as a CUDA graph (lcp.h)."""

    def __init__(self, index: "Index", n: int, Q: int, k: int):
        self._h = ctypes.c_void_p()
        self.index, self.n, self.Q, self.k = index, n, Q, k
        with _on(index.device):
            _check(_lib.lcp_step_create(index.handle, n, Q, k, ctypes.byref(self._h)), "lcp_step_create")

    def run(self, inserts: torch.Tensor, queries: torch.Tensor, out_ids=None, out_lcp=None, stream=None):
        out_ids, out_lcp = _outputs(self.Q, self.k, queries.device, out_ids, out_lcp)
        with _on(queries.device):
            _check(_lib.lcp_step_run(self._h, _ptr(inserts.contiguous()), _ptr(queries.contiguous()),
                                     _ptr(out_ids), _ptr(out_lcp), _stream(stream)), "lcp_step_run")
        return out_ids, out_lcp

    def stats(self):
        r, i = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.lcp_step_stats(self._h, ctypes.byref(r), ctypes.byref(i)), "lcp_step_stats")
        return r.value, i.value

    def close(self):
        if self._h is not None and self._h.value:
            _lib.lcp_step_destroy(self._h)
        self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Session:
    """Serving session over resident indexes (see include/lcp.h).

    submit() takes host tensors (pinned memory keeps it asynchronous) or
    device tensors and returns a ticket; poll() reports LCP_OK / LCP_PENDING / an error code.
    The session keeps references to its indexes and to in-flight buffers.
    """

    def __init__(self, mem_budget: int, max_inflight: int = 64, streams: int = 4,
                 dry_run: bool = False):
        cfg = SessionConfig(mem_budget, max_inflight, streams, 1 if dry_run else 0)
        self._h = ctypes.c_void_p()
        _check(_lib.lcp_session_create(ctypes.byref(cfg), ctypes.byref(self._h)), "lcp_session_create")
        self._indexes = []
        self._live = {}

    def add_index(self, index) -> int:
        slot = ctypes.c_int32()
        h = index.handle if index is not None else ctypes.c_void_p(0)
        _check(_lib.lcp_session_add_index(self._h, h, ctypes.byref(slot)), "lcp_session_add_index")
        self._indexes.append(index)
        return slot.value

    def add_scan(self, tokens: torch.Tensor, vocab: int = 0) -> int:
        """Registers resident tokens ([N, L] device tensor, kept alive here)
        answered by the full scan; returns the slot."""
        tokens = _rows(tokens, device=True)
        slot = ctypes.c_int32()
        _check(_lib.lcp_session_add_scan(self._h, _ptr(tokens), tokens.shape[0], _fmt(tokens, vocab),
                                         ctypes.byref(slot)), "lcp_session_add_scan")
        self._indexes.append(tokens)
        return slot.value

    def submit(self, slot: int, queries, k: int, out_ids=None, out_lcp=None) -> int:
        """Queues a request; returns its ticket.  Raises LcpError (code
        LCP_ERR_BUDGET when the request can never fit the budget)."""
        Q = queries.shape[0] if queries is not None else 0
        on_dev = queries is not None and queries.is_cuda
        if queries is not None:
            queries = _rows(queries, device=on_dev)
        if out_ids is None:
            out_ids = (torch.empty((Q, k), dtype=torch.int32, device=queries.device) if on_dev else
                       torch.empty((Q, k), dtype=torch.int32, pin_memory=torch.cuda.is_available()))
        if out_lcp is None:
            out_lcp = (torch.empty((Q, k), dtype=torch.uint8, device=queries.device) if on_dev else
                       torch.empty((Q, k), dtype=torch.uint8, pin_memory=torch.cuda.is_available()))
        t = ctypes.c_uint64()
        _check(_lib.lcp_session_submit(self._h, slot, _ptr(queries), Q, k, _ptr(out_ids), _ptr(out_lcp),
                                       ctypes.byref(t)), "lcp_session_submit")
        self._live[t.value] = (queries, out_ids, out_lcp)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0) -> int:
        rc = _lib.lcp_session_poll(self._h, ticket, timeout_ms)
        if rc != LCP_PENDING:
            self._live.pop(ticket, None)
        return rc

    def result(self, ticket: int, timeout_ms: int = 10_000):
        """Waits for a ticket and returns its (ids, lcp) host tensors."""
        bufs = self._live.get(ticket)
        rc = self.poll(ticket, timeout_ms)
        if rc != LCP_OK:
            raise LcpError(rc, "lcp_session_poll")
        return bufs[1], bufs[2]

    def replay(self, reqs, timeout_s: float = 120.0):
        """Open-loop replay of ReplayRequest records (see lcp_session_replay).
        Returns (rc, latencies in seconds (numpy), wall seconds)."""
        import numpy as np
        n = len(reqs)
        arr = (ReplayRequest * n)(*reqs)
        lat = (ctypes.c_double * max(n, 1))()
        wall = ctypes.c_double()
        rc = _lib.lcp_session_replay(self._h, arr, n, timeout_s, lat, ctypes.byref(wall))
        return rc, np.ctypeslib.as_array(lat)[:n].copy(), wall.value

    def stats(self) -> dict:
        st = SessionStats()
        _check(_lib.lcp_session_stats(self._h, ctypes.byref(st)), "lcp_session_stats")
        return {n: getattr(st, n) for n, _ in SessionStats._fields_}

    def close(self) -> int:
        rc = LCP_OK
        if self._h is not None and self._h.value:
            rc = _lib.lcp_session_destroy(self._h)
        self._h = None
        self._live.clear()
        return rc

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def raw_lib():
    """The ctypes handle of liblcp.so (for callers marshalling raw pointers)."""
    return _lib
