"""CPU oracle for LCP top-k retrieval -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it; the product path fails loudly when its CUDA extension
is missing instead of falling back here.

The arithmetic lives in ``lcp_oracle.c`` (plain C, see its header for the
definitions it follows: Definitions "LCP Similarity" and "Top-k LCP
Retrieval", Sec. 2.1, and Algorithm 1, Sec. 5.2).  This module compiles it
with gcc and marshals numpy arrays to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcp_oracle.c")
_LIB = os.path.join(_HERE, "liblcp_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.oracle_lcp.argtypes = [vp, vp, i32, i32]
        lib.oracle_lcp.restype = i32
        lib.oracle_topk.argtypes = [vp, i64, i32, i32, vp, i32, vp, vp]
        lib.oracle_topk.restype = i32
        lib.oracle_topk_batch.argtypes = [vp, i64, i32, i32, vp, i64, i32, vp, vp, i32]
        lib.oracle_topk_batch.restype = i32
        lib.oracle_sorted_index.argtypes = [vp, i64, i32, i32, vp, vp]
        lib.oracle_sorted_index.restype = i32
        lib.oracle_topk_bfs.argtypes = [vp, i64, i32, i32, vp, i32, vp, vp]
        lib.oracle_topk_bfs.restype = i32
        lib.oracle_tal_topk.argtypes = [vp, i64, i32, i32, vp, i32, i32, vp, vp]
        lib.oracle_tal_topk.restype = i32
        lib.oracle_topk_wide_batch.argtypes = [vp, i64, i32, i32, vp, i64, i32, vp, vp, i32]
        lib.oracle_topk_wide_batch.restype = i32
        lib.oracle_sorted_index_wide.argtypes = [vp, i64, i32, i32, vp, vp]
        lib.oracle_sorted_index_wide.restype = i32
        _lib = lib
    return _lib


def _rows(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype not in (np.uint8, np.uint16):
        raise TypeError("tokens must be uint8 or uint16, got %s" % a.dtype)
    if a.ndim != 2:
        raise ValueError("tokens must be [n, L]")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def lcp(s: np.ndarray, t: np.ndarray) -> int:
    """LCP(s, t) for two rows of the same token type (Sec. 2.1, Def. LCP)."""
    s = np.ascontiguousarray(s)
    t = np.ascontiguousarray(t, dtype=s.dtype)
    return int(_load().oracle_lcp(_ptr(s), _ptr(t), s.shape[-1], s.itemsize))


def topk(S: np.ndarray, q: np.ndarray, k: int):
    """Top-k of one query: (ids[k] int32, lcp[k] uint8), padded with (-1, 0)."""
    S = _rows(S)
    q = np.ascontiguousarray(q, dtype=S.dtype).reshape(-1)
    ids = np.empty(k, np.int32)
    lc = np.empty(k, np.uint8)
    rc = _load().oracle_topk(_ptr(S), S.shape[0], S.shape[1], S.itemsize, _ptr(q), k,
                             _ptr(ids), _ptr(lc))
    if rc:
        raise ValueError("oracle_topk rejected its arguments (rc=%d)" % rc)
    return ids, lc


def topk_batch(S: np.ndarray, Qs: np.ndarray, k: int, threads: int | None = None):
    """Top-k for every query row: (ids[Q,k] int32, lcp[Q,k] uint8)."""
    S = _rows(S)
    Qs = np.ascontiguousarray(Qs, dtype=S.dtype)
    if Qs.ndim != 2 or Qs.shape[1] != S.shape[1]:
        raise ValueError("queries must be [Q, L] with the dataset's L")
    Q = Qs.shape[0]
    ids = np.empty((Q, k), np.int32)
    lc = np.empty((Q, k), np.uint8)
    if threads is None:
        threads = os.cpu_count() or 1
    rc = _load().oracle_topk_batch(_ptr(S), S.shape[0], S.shape[1], S.itemsize, _ptr(Qs),
                                   Q, k, _ptr(ids), _ptr(lc), threads)
    if rc:
        raise ValueError("oracle_topk_batch rejected its arguments (rc=%d)" % rc)
    return ids, lc


def sorted_index(S: np.ndarray):
    """Sorted order of the items and adjacent-LCP array: (ids[N] int32, H[N] uint8)."""
    S = _rows(S)
    N = S.shape[0]
    ids = np.empty(N, np.int32)
    H = np.empty(N, np.uint8)
    rc = _load().oracle_sorted_index(_ptr(S), N, S.shape[1], S.itemsize, _ptr(ids), _ptr(H))
    if rc:
        raise ValueError("oracle_sorted_index rejected its arguments (rc=%d)" % rc)
    return ids, H


def _per_query(fn, S, Qs, k, *extra):
    S = _rows(S)
    Qs = np.ascontiguousarray(Qs, dtype=S.dtype)
    if Qs.ndim != 2 or Qs.shape[1] != S.shape[1]:
        raise ValueError("queries must be [Q, L] with the dataset's L")
    Q = Qs.shape[0]
    ids = np.empty((Q, k), np.int32)
    lc = np.empty((Q, k), np.uint8)
    for i in range(Q):
        q = np.ascontiguousarray(Qs[i])
        rc = fn(_ptr(S), S.shape[0], S.shape[1], S.itemsize, _ptr(q), k, *extra,
                _ptr(ids[i]), _ptr(lc[i]))
        if rc:
            raise ValueError("oracle rejected its arguments (rc=%d)" % rc)
    return ids, lc


def topk_bfs(S: np.ndarray, Qs: np.ndarray, k: int):
    """Algorithms 3 + 4 literally (BFS order within the deepest node's
    subtree), per query row: (ids[Q,k] int32, lcp[Q,k] uint8)."""
    return _per_query(_load().oracle_topk_bfs, S, Qs, k)


def tal_topk(S: np.ndarray, Qs: np.ndarray, k: int, d: int):
    """TAL bucket scan at prefix depth d, per query row: the top k of the
    items sharing the query's first d symbols, padded."""
    return _per_query(_load().oracle_tal_topk, S, Qs, k, d)



def topk_wide(S: np.ndarray, Qs: np.ndarray, k: int, threads: int | None = None):
    """Top-k for every query row over rows of any length L <= 65535 (the
    paper's sustained shape has L = 256): (ids[Q,k] int32, lcp[Q,k] uint16)."""
    S = _rows(S)
    Qs = np.ascontiguousarray(Qs, dtype=S.dtype)
    if Qs.ndim != 2 or Qs.shape[1] != S.shape[1]:
        raise ValueError("queries must be [Q, L] with the dataset's L")
    Q = Qs.shape[0]
    ids = np.empty((Q, k), np.int32)
    lc = np.empty((Q, k), np.uint16)
    if threads is None:
        threads = os.cpu_count() or 1
    rc = _load().oracle_topk_wide_batch(_ptr(S), S.shape[0], S.shape[1], S.itemsize, _ptr(Qs), Q, k,
                                        _ptr(ids), _ptr(lc), threads)
    if rc:
        raise ValueError("oracle_topk_wide_batch rejected its arguments (rc=%d)" % rc)
    return ids, lc


def sorted_index_wide(S: np.ndarray):
    """Sorted order and adjacent-LCP array for rows of any length:
    (ids[N] int32, H[N] uint16)."""
    S = _rows(S)
    N = S.shape[0]
    ids = np.empty(N, np.int32)
    H = np.empty(N, np.uint16)
    rc = _load().oracle_sorted_index_wide(_ptr(S), N, S.shape[1], S.itemsize, _ptr(ids), _ptr(H))
    if rc:
        raise ValueError("oracle_sorted_index_wide rejected its arguments (rc=%d)" % rc)
    return ids, H
