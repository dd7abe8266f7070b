"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws token sequences, queries and request streams.  It holds
none of the retrieval method's arithmetic (no LCP, no sorting of sequences, no
top-k), so both the CPU oracle and the CUDA library can consume its output.

Randomness is counter based: every draw is ``splitmix64`` (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied
to a key built from (seed, stream, item, position), so any row can be
regenerated on its own and results do not depend on batch order.

Workloads (the paper's own inputs are synthetic; these follow its shapes):

* ``tree_u8``      -- small prefix-tree set: alphabet 16, L=16 uint8; a complete
  4-ary tree over the first 8 positions (each node's 4 symbols are a seeded
  4-subset of the alphabet), the last 8 positions uniform.
* ``zipf_prefix``  -- uint16 tokens; position j is Zipf(s) over ranks 1..V,
  mapped through a per-prefix seeded permutation pi_h(r) = (a_h (r-1) + b_h)
  mod V (a_h odd, V a power of two, so pi_h is a bijection); h_0 comes from the
  seed and h_{j+1} = splitmix64(h_j XOR (token_j + 1)).  Popular prefixes are
  therefore heavily shared.
* query mix        -- half copies of a uniformly chosen stored row whose suffix
  from a uniform cut depth c in [0, L] is re-drawn from the same generator
  (continuing from the kept prefix), half fresh draws.
* ``gnc_stream``   -- 1,000 sensors: [type < 16, subsystem < 64, six decimal
  digits of a random-walk value in [0, 999999], most significant first], L=8.
* ``serving_mix``  -- Poisson request arrivals, log-uniform batch sizes in
  [1, 4096], k drawn from {1, 10, 100}, index drawn uniformly.
* ``sustained2m_L256`` -- the sustained shape: zipf_prefix rows of 256
  tokens; copies keep a fixed prefix of 128 tokens (prefix_len).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_U64 = np.uint64
_GOLDEN = 0x9E3779B97F4A7C15

# Stream identifiers: independent sub-streams of one seed.
STREAM_ROWS = 1
STREAM_QMIX = 2
STREAM_QTOK = 3
STREAM_TREE = 4
STREAM_GNC = 5
STREAM_SERVE = 6
STREAM_PERM = 7
STREAM_UNIFORM = 8


def splitmix64(x):
    """splitmix64 finaliser over a uint64 array (wrapping arithmetic)."""
    x = np.asarray(x, dtype=_U64)
    with np.errstate(over="ignore"):
        z = x + _U64(_GOLDEN)
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        return z ^ (z >> _U64(31))


def rand_u64(seed: int, stream: int, a, b=0):
    """Counter-based 64-bit draw keyed by (seed, stream, a, b)."""
    a = np.asarray(a, dtype=_U64)
    b = np.asarray(b, dtype=_U64)
    key = splitmix64(splitmix64(_U64(seed & 0xFFFFFFFFFFFFFFFF)) ^ _U64(stream))
    with np.errstate(over="ignore"):
        return splitmix64(splitmix64(key + a) ^ (b * _U64(0xD6E8FEB86659FD93)))


def stream_key(seed: int, stream: int) -> int:
    """The 64-bit key of (seed, stream) used by rand_u64."""
    return int(splitmix64(splitmix64(_U64(seed & 0xFFFFFFFFFFFFFFFF)) ^ _U64(stream)))


def rand_uniform(seed: int, stream: int, a, b=0):
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (rand_u64(seed, stream, a, b) >> _U64(11)).astype(np.float64) * (1.0 / (1 << 53))


def _prefix_root(seed: int) -> np.uint64:
    return splitmix64(_U64((seed * 0x2545F4914F6CDD1D + 0xA0761D6478BD642F) & 0xFFFFFFFFFFFFFFFF))


def _chain(h, tok):
    """Prefix hash update h_{j+1} = splitmix64(h_j XOR (token_j + 1))."""
    return splitmix64(np.asarray(h, _U64) ^ (np.asarray(tok, _U64) + _U64(1)))


class Zipf:
    """Zipf(s) over ranks 1..V by double-precision inverse CDF."""

    def __init__(self, V: int, s: float):
        w = np.arange(1, V + 1, dtype=np.float64) ** (-s)
        self.cdf = np.cumsum(w) / w.sum()
        self.V = V

    def rank0(self, u):
        """0-based rank r-1 for uniforms u in [0, 1)."""
        r = np.searchsorted(self.cdf, u, side="right")
        return np.minimum(r, self.V - 1).astype(np.int64)


def _perm_token(h, r0, V: int):
    """pi_h applied to 0-based rank r0: (a_h * r0 + b_h) mod V, a_h odd."""
    a = splitmix64(h) | _U64(1)
    b = splitmix64(h ^ _U64(0xD1B54A32D192ED03))
    m = _U64(V - 1)
    with np.errstate(over="ignore"):
        return ((a * np.asarray(r0, _U64) + b) & m).astype(np.int64)


# --------------------------------------------------------------------------
# C fast path (workloads/gen.c): the same draws, bit for bit
# --------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SO = os.path.join(_HERE, "libgen.so")
_gen = None


def build_gen(force: bool = False) -> str:
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_GEN_SO) or os.path.getmtime(_GEN_SO) < os.path.getmtime(src):
        tmp = _GEN_SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp,
                               src])
        os.replace(tmp, _GEN_SO)
    return _GEN_SO


def _gen_lib():
    global _gen
    if _gen is None:
        lib = ctypes.CDLL(build_gen())
        vp, i64, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64
        lib.gen_zipf_prefix.argtypes = [vp, i64, i64, i64, vp, u64, u64, i64, vp, vp, vp,
                                        ctypes.c_int]
        lib.gen_zipf_prefix.restype = None
        _gen = lib
    return _gen


def _c_zipf(n, L, V, cdf, key, h0, item_offset, S=None, src=None, cut=None):
    out = np.empty((n, L), np.uint16)
    cdf = np.ascontiguousarray(cdf, np.float64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None
    if S is not None:
        S = np.ascontiguousarray(S, np.uint16)
        src = np.ascontiguousarray(src, np.int64)
        cut = np.ascontiguousarray(cut, np.int64)
    _gen_lib().gen_zipf_prefix(p(out), n, L, V, p(cdf), key, int(h0), item_offset, p(S), p(src),
                               p(cut), min(os.cpu_count() or 1, 64))
    return out


# --------------------------------------------------------------------------
# stored sequences
# --------------------------------------------------------------------------

def zipf_prefix_rows(N: int, L: int, V: int, s: float, seed: int, stream: int = STREAM_ROWS,
                     item_offset: int = 0, impl: str = "c") -> np.ndarray:
    """N rows of L uint16 tokens, Zipf(s) per position, prefix-conditioned."""
    if V & (V - 1) or V > 65536:
        raise ValueError("V must be a power of two <= 65536")
    z = Zipf(V, s)
    if impl == "c":
        return _c_zipf(N, L, V, z.cdf, stream_key(seed, stream), _prefix_root(seed), item_offset)
    out = np.empty((N, L), np.uint16)
    items = np.arange(item_offset, item_offset + N, dtype=np.uint64)
    h = np.full(N, _prefix_root(seed), _U64)
    for j in range(L):
        u = rand_uniform(seed, stream, items, j)
        t = _perm_token(h, z.rank0(u), V)
        out[:, j] = t
        h = _chain(h, t)
    return out


def tree_rows(N: int, seed: int, L: int = 16, depth: int = 8, branch: int = 4,
              sigma: int = 16, stream: int = STREAM_TREE, item_offset: int = 0) -> np.ndarray:
    """Rows of a complete `branch`-ary prefix tree over the first `depth`
    positions (each node's children are a seeded `branch`-subset of the
    alphabet); later positions uniform over the alphabet.  uint8 tokens."""
    out = np.empty((N, L), np.uint8)
    items = np.arange(item_offset, item_offset + N, dtype=np.uint64)
    h = np.full(N, _prefix_root(seed), _U64)
    for j in range(L):
        u = rand_uniform(seed, stream, items, j)
        if j < depth:
            c = np.minimum((u * branch).astype(np.int64), branch - 1)
            t = _perm_token(h, c, sigma)
        else:
            t = np.minimum((u * sigma).astype(np.int64), sigma - 1)
        out[:, j] = t
        h = _chain(h, t)
    return out


# --------------------------------------------------------------------------
# queries
# --------------------------------------------------------------------------

def _mix_plan(Q: int, N: int, L: int, seed: int, item_offset: int = 0, fixed_cut: int | None = None):
    items = np.arange(item_offset, item_offset + Q, dtype=np.uint64)
    is_copy = rand_uniform(seed, STREAM_QMIX, items, 0) < 0.5
    if N == 0:
        is_copy[:] = False
    src = np.minimum((rand_uniform(seed, STREAM_QMIX, items, 1) * max(N, 1)).astype(np.int64),
                     max(N - 1, 0))
    cut = np.minimum((rand_uniform(seed, STREAM_QMIX, items, 2) * (L + 1)).astype(np.int64), L)
    if fixed_cut is not None:
        cut[:] = min(fixed_cut, L)
    cut = np.where(is_copy, cut, 0)
    return items, is_copy, src, cut


def zipf_prefix_queries(S: np.ndarray, Q: int, V: int, s: float, seed: int,
                        item_offset: int = 0, impl: str = "c", fixed_cut: int | None = None) -> np.ndarray:
    """Query mix over a zipf_prefix dataset S (see module docstring); with
    `fixed_cut`, every copy keeps exactly its first `fixed_cut` tokens."""
    N, L = S.shape
    z = Zipf(V, s)
    items, is_copy, src, cut = _mix_plan(Q, N, L, seed, item_offset, fixed_cut)
    if impl == "c":
        Sx = S if N > 0 else np.zeros((1, L), np.uint16)
        return _c_zipf(Q, L, V, z.cdf, stream_key(seed, STREAM_QTOK), _prefix_root(seed),
                       item_offset, Sx, src, cut)
    out = np.empty((Q, L), np.uint16)
    h = np.full(Q, _prefix_root(seed), _U64)
    src_rows = S[src] if N > 0 else np.zeros((Q, L), np.uint16)
    for j in range(L):
        keep = j < cut
        u = rand_uniform(seed, STREAM_QTOK, items, j)
        drawn = _perm_token(h, z.rank0(u), V)
        t = np.where(keep, src_rows[:, j].astype(np.int64), drawn)
        out[:, j] = t
        h = _chain(h, t)
    return out


def tree_queries(S: np.ndarray, Q: int, seed: int, sigma: int = 16,
                 item_offset: int = 0) -> np.ndarray:
    """Query mix for tree_rows: copies with the suffix from a uniform cut
    re-drawn uniformly over the alphabet, and uniform random rows."""
    N, L = S.shape
    items, is_copy, src, cut = _mix_plan(Q, N, L, seed, item_offset)
    out = np.empty((Q, L), np.uint8)
    src_rows = S[src] if N > 0 else np.zeros((Q, L), np.uint8)
    for j in range(L):
        u = rand_uniform(seed, STREAM_QTOK, items, j)
        drawn = np.minimum((u * sigma).astype(np.int64), sigma - 1)
        out[:, j] = np.where(j < cut, src_rows[:, j].astype(np.int64), drawn)
    return out


# --------------------------------------------------------------------------
# GNC-style sensor stream
# --------------------------------------------------------------------------

class GncStream:
    """1,000 sensors (by default); step t yields one reading per sensor.

    Reading tokens: [type, subsystem, d5, d4, d3, d2, d1, d0] (uint16, L=8),
    where d5..d0 are the decimal digits of a random-walk value v in
    [0, 999999]; v <- clamp(v + U{-500..500}).  Ids of step t's readings are
    t * sensors + i.
    """

    L = 8

    def __init__(self, sensors: int = 1000, seed: int = 5):
        self.sensors, self.seed = sensors, seed
        i = np.arange(sensors, dtype=np.uint64)
        self.type = np.minimum((rand_uniform(seed, STREAM_GNC, i, 0) * 16).astype(np.int64), 15)
        self.sub = np.minimum((rand_uniform(seed, STREAM_GNC, i, 1) * 64).astype(np.int64), 63)
        self.v = np.minimum((rand_uniform(seed, STREAM_GNC, i, 2) * 1_000_000).astype(np.int64),
                            999_999)
        self.t = 0

    def step(self) -> np.ndarray:
        if self.t > 0:
            i = np.arange(self.sensors, dtype=np.uint64)
            d = np.minimum((rand_uniform(self.seed, STREAM_GNC, i, 3 + self.t) * 1001)
                           .astype(np.int64), 1000) - 500
            self.v = np.clip(self.v + d, 0, 999_999)
        self.t += 1
        out = np.empty((self.sensors, self.L), np.uint16)
        out[:, 0] = self.type
        out[:, 1] = self.sub
        v = self.v.copy()
        for j in range(7, 1, -1):
            out[:, j] = v % 10
            v //= 10
        return out


# --------------------------------------------------------------------------
# serving request stream
# --------------------------------------------------------------------------

SERVING_INDEXES = ((1_000, 16), (10_000, 16), (100_000, 32), (500_000, 32),
                   (1_000_000, 64), (2_000_000, 64))


def serving_requests(n_requests: int, rate_per_s: float, n_indexes: int, seed: int,
                     max_q: int = 4096, ks=(1, 10, 100)):
    """Open-loop Poisson request stream.

    Returns dict of arrays: arrival_s (float64, cumulative), n_queries
    (log-uniform in [1, max_q]), k, index.
    """
    r = np.arange(n_requests, dtype=np.uint64)
    gaps = -np.log1p(-rand_uniform(seed, STREAM_SERVE, r, 0)) / rate_per_s
    n = np.floor(np.exp(rand_uniform(seed, STREAM_SERVE, r, 1) * math.log(max_q + 1)))
    n = np.clip(n.astype(np.int64), 1, max_q)
    k = np.asarray(ks, np.int64)[np.minimum((rand_uniform(seed, STREAM_SERVE, r, 2) * len(ks))
                                            .astype(np.int64), len(ks) - 1)]
    idx = np.minimum((rand_uniform(seed, STREAM_SERVE, r, 3) * n_indexes).astype(np.int64),
                     n_indexes - 1)
    return {"arrival_s": np.cumsum(gaps), "n_queries": n, "k": k, "index": idx}


def uniform_rows(n: int, L: int, V: int, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """n rows of L tokens, each uniform over 0..V-1 (V <= 65536), drawn
    counter-based per (row, position); uint8 when V <= 256, else uint16."""
    dt = np.uint8 if V <= 256 else np.uint16
    out = np.empty((n, L), dt)
    pos = np.arange(L, dtype=_U64)
    for a in range(0, n, chunk):
        rows = np.arange(a, min(n, a + chunk), dtype=_U64)
        r = rand_u64(seed, STREAM_UNIFORM, rows[:, None], pos[None, :])
        out[a:a + len(rows)] = (r % _U64(V)).astype(dt)
    return out


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

WORKLOADS = {
    "tree16_u8": dict(N=10_000, L=16, token_bytes=1, vocab=16, Q=1_000, k=10, seed=1),
    "zipf500k_L32": dict(N=500_000, L=32, token_bytes=2, vocab=1024, s=1.1, Q=100_000, k=32,
                         seed=2),
    "zipf2m_L64": dict(N=2_000_000, L=64, token_bytes=2, vocab=32768, s=1.05, Q=1_000_000,
                       k=100, seed=3),
    "serving6": dict(vocab=32768, s=1.05, rate=20_000.0, seed=4),
    "gnc1000": dict(sensors=1000, steps=1000, L=8, token_bytes=2, k=5, seed=5),
    # the paper's TAL benchmark shape: 20M items, 256 prefix buckets (uniform
    # first token over 256 values, bucket depth 1), 10,000 queries
    "tal20m": dict(N=20_000_000, L=16, token_bytes=1, vocab=256, depth=1, Q=10_000, k=10, seed=6),
    # the paper's sustained shape: top-1 over 2M sequences of max_len 256,
    # one query at a time; copies keep their first prefix_len = 128 tokens
    "sustained2m_L256": dict(N=2_000_000, L=256, token_bytes=2, vocab=32768, s=1.05, Q=100_000, k=1,
                             seed=7, prefix_len=128),
}


def make_dataset(name: str, N: int | None = None, Q: int | None = None):
    """(S, queries, k) for the static workloads, optionally shrunk to N / Q."""
    w = WORKLOADS[name]
    N = w["N"] if N is None else N
    Q = w["Q"] if Q is None else Q
    if name == "tree16_u8":
        S = tree_rows(N, w["seed"], L=w["L"])
        return S, tree_queries(S, Q, w["seed"]), w["k"]
    S = zipf_prefix_rows(N, w["L"], w["vocab"], w["s"], w["seed"])
    return S, zipf_prefix_queries(S, Q, w["vocab"], w["s"], w["seed"], fixed_cut=w.get("prefix_len")), w["k"]
