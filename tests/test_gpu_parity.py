"""GPU parity: the CUDA paths against the CPU oracle, bit for bit.

Every comparison is exact (ids and LCPs are integers; the answer is unique
because the key (-LCP, id) is).  Inputs are seeded; the oracle never sees GPU
output.  Small cases are compared element by element on every query; the
full-size workloads are compared on sampled queries through the oracle and on
every query between the indexed path and the full scan.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lcp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_04936_b300 as P
    return P


def dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a).cuda()


def host(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a)


def indexed(lcp, S, Qs, k, max_k=None, shape=None):
    """Indexed search; `shape` = (qpw, locate_warp) forces a launch shape
    (qpw 0: the fused kernel, else locate + answer + fill)."""
    idx = lcp.lcp_index_build(dev(S), max_k=max_k or max(k, 1))
    if shape is not None and len(Qs):
        lcp.lcp_set_search_shape(idx, len(Qs), k, shape[0], shape[1])
    ids, lc = lcp.lcp_topk_batch(idx, dev(Qs), k)
    torch.cuda.synchronize()
    assert lcp.lcp_index_sync(idx) == 0
    out = ids.cpu().numpy(), lc.cpu().numpy()
    idx.close()
    return out


def scan(lcp, S, Qs, k):
    ids, lc = lcp.lcp_scan_topk(dev(S), dev(Qs), k)
    torch.cuda.synchronize()
    assert lcp.lcp_device_status() == 0
    return ids.cpu().numpy(), lc.cpu().numpy()


def assert_same(got, want, what):
    gi, gl = got
    wi, wl = want
    if not (np.array_equal(gi, wi) and np.array_equal(gl, wl)):
        bad = np.nonzero((gi != wi).any(1) | (gl != wl).any(1))[0]
        r = bad[0]
        raise AssertionError("%s: %d/%d queries differ; first q=%d\n got ids %s lcp %s\nwant ids %s lcp %s"
                             % (what, len(bad), len(gi), r, gi[r][:16], gl[r][:16], wi[r][:16],
                                wl[r][:16]))


def _prefixy(rng, N, L, sigma, dt, share=4):
    if N == 0:
        return np.zeros((0, L), dt)
    base = rng.integers(0, sigma, size=(max(N // share, 1), L))
    rows = base[rng.integers(0, base.shape[0], N)].copy()
    cut = rng.integers(0, L + 1, N)
    for i in range(N):
        rows[i, cut[i]:] = rng.integers(0, sigma, L - cut[i])
    return rows.astype(dt)


def _queries(rng, S, Q, sigma, dt):
    N, L = S.shape
    out = rng.integers(0, sigma, size=(Q, L)).astype(dt)
    if N:
        src = S[rng.integers(0, N, Q)]
        cut = rng.integers(0, L + 1, Q)
        for i in range(Q):
            if i % 2 == 0:
                out[i, :cut[i]] = src[i, :cut[i]]
    if Q > 2:
        out[0] = 0  # below every row
        out[1] = np.iinfo(dt).max  # above every row
    return out


CASES = [
    # N, L, token_bytes, sigma, k
    (1, 4, 1, 3, 1),
    (2, 4, 1, 3, 5),
    (37, 3, 1, 2, 10),
    (100, 7, 1, 4, 32),
    (129, 5, 2, 6, 128),
    (1000, 16, 1, 16, 10),
    (1000, 9, 2, 3, 100),
    (4097, 12, 2, 5, 64),
    (5000, 33, 2, 4, 100),
    (20000, 8, 1, 2, 128),   # tiny alphabet: enormous tie levels
    (3000, 255, 1, 2, 17),   # L = 255, uint8
    (3000, 10, 1, 3, 80),    # K = 96: sparse table merged in shared memory
    (20000, 24, 1, 2, 50),   # mid-size tie groups, word 1 ties resolved on word 2
    (700, 255, 2, 3, 40),    # L = 255, uint16 (64 packed words)
]


@pytest.mark.parametrize("N,L,tb,sigma,k", CASES)
def test_small_cases_indexed_and_scan_match_oracle(lcp, N, L, tb, sigma, k):
    rng = np.random.default_rng(N * 31 + L * 7 + tb)
    dt = np.uint8 if tb == 1 else np.uint16
    S = _prefixy(rng, N, L, sigma, dt)
    Qs = _queries(rng, S, 300, sigma, dt)
    want = oracle.topk_batch(S, Qs, k)
    assert_same(indexed(lcp, S, Qs, k), want, "indexed")  # small batch: the fused kernel
    assert_same(indexed(lcp, S, Qs, k, shape=(1, 1)), want, "indexed, three kernels")
    assert_same(indexed(lcp, S, Qs, k, shape=(8, 0)), want, "indexed, three kernels, lane locate")
    assert_same(indexed(lcp, S, Qs, k, shape=(4, 2)), want, "indexed, three kernels, staged top levels")
    assert_same(scan(lcp, S, Qs, k), want, "scan")


@pytest.mark.parametrize("N,L,tb,sigma", [(1, 3, 1, 2), (500, 4, 1, 3), (10000, 16, 1, 16),
                                          (50000, 32, 2, 7), (3000, 255, 2, 2), (70000, 5, 1, 2),
                                          (30000, 16, 2, 5),    # 4 words: 8 rows per warp step
                                          (20000, 48, 2, 3),    # 12 words: gather and H separately
                                          (20000, 16, 1, 2),    # ~78-row tie groups, ties on word 1 too
                                          (20000, 12, 2, 3)])   # ~250-row groups, later words decide
def test_sorted_index_matches_oracle(lcp, N, L, tb, sigma):
    rng = np.random.default_rng(N + L)
    dt = np.uint8 if tb == 1 else np.uint16
    S = _prefixy(rng, N, L, sigma, dt)
    idx = lcp.lcp_index_build(dev(S), max_k=8)
    ids, H = lcp.lcp_index_export(idx)
    torch.cuda.synchronize()
    assert lcp.lcp_index_sync(idx) == 0
    w_ids, w_H = oracle.sorted_index(S)
    assert np.array_equal(ids.cpu().numpy(), w_ids)
    assert np.array_equal(H.cpu().numpy(), w_H)


def test_sorted_index_many_superblocks(lcp):
    """6,000,000 rows: the build's radix passes run 2,930 tiles, so each
    scatter CTA adds up 92 superblock sums (three rounds of its 32-wide
    loop) before its own superblock's tiles; every digit byte of word 0
    varies (uint16 tokens below 4,096) and rows repeat (ties broken by id)."""
    N, L = 6_000_000, 4
    rng = np.random.default_rng(6)
    S = rng.integers(0, 4096, size=(N, L)).astype(np.uint16)
    S[1::5] = S[rng.integers(0, N, len(S[1::5]))]  # duplicate rows
    idx = lcp.lcp_index_build(dev(S), max_k=8)
    ids, H = lcp.lcp_index_export(idx)
    torch.cuda.synchronize()
    assert lcp.lcp_index_sync(idx) == 0
    idx.close()
    w_ids, w_H = oracle.sorted_index(S)
    assert np.array_equal(ids.cpu().numpy(), w_ids)
    assert np.array_equal(H.cpu().numpy(), w_H)


def test_direct_build_equals_graph_build(lcp):
    """lcp_build_graph(0): the build's kernels launched one by one (what
    per-kernel timing brackets) give the same sorted ids and H as the graph
    replay, and answers stay the oracle's."""
    rng = np.random.default_rng(31)
    S = _prefixy(rng, 30000, 16, 5, np.uint16)
    Qs = _queries(rng, S, 200, 5, np.uint16)
    g = lcp.lcp_index_build(dev(S), max_k=20)
    g_ids, g_H = lcp.lcp_index_export(g)
    lcp.lcp_build_graph(False)
    try:
        d = lcp.lcp_index_build(dev(S), max_k=20)
        d_ids, d_H = lcp.lcp_index_export(d)
        got = lcp.lcp_topk_batch(d, dev(Qs), 20)
        torch.cuda.synchronize()
        assert lcp.lcp_index_sync(d) == 0
    finally:
        lcp.lcp_build_graph(True)
    assert torch.equal(g_ids, d_ids) and torch.equal(g_H, d_H)
    assert_same((got[0].cpu().numpy(), got[1].cpu().numpy()), oracle.topk_batch(S, Qs, 20), "direct build")
    g.close()
    d.close()


def test_edge_cases(lcp):
    # empty dataset: all padding
    S = np.zeros((0, 6), np.uint8)
    Qs = np.ones((5, 6), np.uint8)
    for got in (indexed(lcp, S, Qs, 4), scan(lcp, S, Qs, 4)):
        assert (got[0] == -1).all() and (got[1] == 0).all()
    # all identical rows, queries equal / off in the last token / off in the first
    S = np.full((3000, 10), 7, np.uint16)
    Qs = np.full((3, 10), 7, np.uint16)
    Qs[1, -1] = 8
    Qs[2, 0] = 6
    for k in (1, 50, 128):
        want = oracle.topk_batch(S, Qs, k)
        assert_same(indexed(lcp, S, Qs, k), want, "indexed identical rows")
        assert_same(scan(lcp, S, Qs, k), want, "scan identical rows")
    # rows differing only in the last token; token values at the top of the range
    S = np.tile(np.array([[0xFFFF] * 6], np.uint16), (300, 1))
    S[:, -1] = np.arange(300, dtype=np.uint16)[::-1] * 200
    Qs = S[::7].copy()
    want = oracle.topk_batch(S, Qs, 20)
    assert_same(indexed(lcp, S, Qs, 20), want, "indexed last-token")
    assert_same(scan(lcp, S, Qs, 20), want, "scan last-token")
    # k larger than N
    rng = np.random.default_rng(1)
    S = rng.integers(0, 3, size=(9, 5)).astype(np.uint8)
    Qs = rng.integers(0, 3, size=(40, 5)).astype(np.uint8)
    want = oracle.topk_batch(S, Qs, 30)
    assert_same(indexed(lcp, S, Qs, 30), want, "indexed k>N")
    assert_same(scan(lcp, S, Qs, 30), want, "scan k>N")


def test_tree16_u8_full(lcp):
    """The small prefix-tree workload in full: every query, both paths."""
    S, Qs, k = W.make_dataset("tree16_u8")
    want = oracle.topk_batch(S, Qs, k)
    assert_same(indexed(lcp, S, Qs, k), want, "indexed tree16")
    assert_same(scan(lcp, S, Qs, k), want, "scan tree16")


@pytest.mark.parametrize("N,L,tb,sigma,k", [(5000, 7, 1, 3, 20),      # rows not 8-byte aligned
                                             (20000, 16, 2, 5, 100),
                                             (3000, 255, 1, 2, 17),
                                             (2000, 12, 2, 2, 1024),    # k = the largest full-scan k
                                             (40000, 12, 2, 2, 1024),   # slices > k rows: logs compacted
                                             (300, 5, 1, 2, 1000)])     # k > N
def test_scan_batch_paths_agree(lcp, N, L, tb, sigma, k):
    """Full scan: one batch of 8,200 queries (per-thread logs), the same
    queries in batches of 410 (threshold selection, batches <= 1,024) and one
    query at a time (the walk reads word 0 straight from the rows) give the
    same bytes, and match the oracle on a sample."""
    rng = np.random.default_rng(N * 13 + L * 5 + k)
    dt = np.uint8 if tb == 1 else np.uint16
    S = _prefixy(rng, N, L, sigma, dt)
    Qs = _queries(rng, S, 8200, sigma, dt)
    big = scan(lcp, S, Qs, k)
    parts = [scan(lcp, S, Qs[i:i + 410], k) for i in range(0, len(Qs), 410)]
    small = np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])
    assert_same(small, big, "scan: batches of 410 vs one batch of 8,200")
    pick = np.sort(rng.choice(len(Qs), 40, replace=False))
    want = oracle.topk_batch(S, Qs[pick], k)
    assert_same((big[0][pick], big[1][pick]), want, "scan vs oracle (sample)")
    for j in range(8):
        i = pick[j]
        assert_same(scan(lcp, S, Qs[i:i + 1], k), (want[0][j:j + 1], want[1][j:j + 1]), "scan, one query")


@pytest.mark.parametrize("Q,L,tb", [(1, 16, 2), (5, 16, 2), (33, 16, 2), (70, 32, 2), (257, 16, 1),
                                     (40, 12, 2), (3, 8, 2), (64, 16, 1), (200, 3, 1), (190, 2, 1),
                                     (160, 1, 2), (170, 16, 2), (300, 5, 2), (400, 12, 2), (700, 16, 2),
                                     (500, 9, 1)])
def test_scan_selection_batch_shapes(lcp, Q, L, tb):
    """Threshold selection at batch sizes that split a count CTA's 8 warps
    differently: one chunk of 32 queries over 8 row parts (Q <= 32), 3 chunks
    over 2 parts (70), more chunks than warps (257); rows fed by tensor copies
    (16-byte multiples) or by plain loads (24-byte rows); granules ragged at
    the end (N not a multiple of 256).  From 160 queries the full granules
    are sorted by word 0 and searched, including rows shorter than the four
    levels counted per granule (L = 1, 2, 3; L = 5 uint16 has a one-token
    word 1) and rows fed by plain loads (12 uint16 tokens, 24-byte rows).
    The answer CTAs run 1,024, 512 or 256 threads as the batch grows (500
    and 700 queries: 256)."""
    rng = np.random.default_rng(Q * 7 + L + tb)
    dt = np.uint8 if tb == 1 else np.uint16
    S = _prefixy(rng, 30011, L, 4, dt)
    Qs = _queries(rng, S, Q, 4, dt)
    for k in (1, 50, 300):
        assert_same(scan(lcp, S, Qs, k), oracle.topk_batch(S, Qs, k), "scan Q=%d k=%d" % (Q, k))


def test_scan_shared_prefix_beyond_list(lcp):
    """More rows share a query's first 8 tokens than the selection keeps per
    query (6,000 of 9,000 rows): the exact pass over all rows in id order;
    beside it queries answered from the list and by the walk."""
    rng = np.random.default_rng(77)
    S = rng.integers(0, 3, size=(9000, 16)).astype(np.uint16)
    S[:6000, :8] = 5
    Qs = rng.integers(0, 3, size=(6, 16)).astype(np.uint16)
    Qs[:3, :8] = 5
    Qs[1, 8:] = S[4321, 8:]
    Qs[3] = S[8500]
    for k in (1, 10, 100, 1000):
        assert_same(scan(lcp, S, Qs, k), oracle.topk_batch(S, Qs, k), "scan shared prefix k=%d" % k)
        assert_same(scan(lcp, S, Qs[1:2], k), oracle.topk_batch(S, Qs[1:2], k), "one query k=%d" % k)


@pytest.mark.parametrize("tb", [1, 2])
def test_depth2_bucket_tables(lcp, tb):
    """First tokens with at least 4,096 rows get depth-2 bucket tables (runs
    of (first, second token)); queries whose d* is 2 read their tie interval
    from them.  Three big first tokens, second tokens at both ends of the
    range and in between, against the oracle (and an index with insert
    capacity, which has no tables)."""
    rng = np.random.default_rng(23 + tb)
    dt = np.uint8 if tb == 1 else np.uint16
    top = np.iinfo(dt).max
    N, L = 30000, 12
    S = rng.integers(0, 6, size=(N, L)).astype(dt)
    S[:, 0] = rng.choice(np.array([3, 7, top], dt), N, p=[0.45, 0.35, 0.2])
    S[:, 1] = rng.choice(np.array([0, 1, 2, top - 1, top], dt), N)
    Qs = S[rng.integers(0, N, 400)].copy()
    Qs[:, 2:] = rng.integers(6, 9, size=(400, L - 2))  # LCP exactly 2 with their source rows
    Qs[:40, 1] = 5  # second token absent: d* = 1
    for k in (5, 100):
        want = oracle.topk_batch(S, Qs, k)
        assert_same(indexed(lcp, S, Qs, k), want, "indexed depth-2 k=%d" % k)
        assert_same(indexed(lcp, S, Qs, k, shape=(8, 0)), want, "indexed depth-2, three kernels k=%d" % k)
    idx = lcp.lcp_index_build(dev(S), max_k=100, capacity=N + 100)
    ids, lc = lcp.lcp_topk_batch(idx, dev(Qs), 100)
    torch.cuda.synchronize()
    assert_same((ids.cpu().numpy(), lc.cpu().numpy()), oracle.topk_batch(S, Qs, 100), "insertable index")
    idx.close()


def test_index_past_2_pow_24_rows(lcp):
    """An index of more than 2^24 rows takes the searches' 64-bit sort keys
    (24 bits no longer hold an id): the fused small-batch kernel and the
    three-kernel path, both against the oracle on dense duplicates and ties."""
    N, L, k = (1 << 24) + 300_000, 6, 20
    rng = np.random.default_rng(24)
    S = rng.integers(0, 16, size=(N, L)).astype(np.uint8)  # 16^6 ~ N: many duplicate rows
    Qs = np.concatenate([S[rng.integers(0, N, 3000)], rng.integers(0, 16, size=(3000, L)).astype(np.uint8)])
    Qs[::7, 3:] = rng.integers(0, 16, size=(len(Qs[::7]), L - 3))
    idx = lcp.lcp_index_build(dev(S), max_k=k)
    small = lcp.lcp_topk_batch(idx, dev(Qs[:64]), k)      # fused kernel
    large = lcp.lcp_topk_batch(idx, dev(Qs), k)           # locate + answer + fill
    torch.cuda.synchronize()
    assert lcp.lcp_index_sync(idx) == 0
    idx.close()
    want = oracle.topk_batch(S, Qs[:64], k)
    assert_same((small[0].cpu().numpy(), small[1].cpu().numpy()), want, "fused, N > 2^24")
    pick = np.sort(rng.choice(len(Qs), 64, replace=False))
    want = oracle.topk_batch(S, Qs[pick], k)
    got = large[0].cpu().numpy()[pick], large[1].cpu().numpy()[pick]
    assert_same(got, want, "three kernels, N > 2^24")


def test_insert_equals_rebuild_and_answers(lcp):
    """GNC stream: merge-insert 1,000 readings per step into an index that
    grows from empty; after every step the sorted order and H equal a fresh
    build of everything inserted, and the step's queries match the oracle."""
    g = W.GncStream(sensors=1000, seed=5)
    idx = lcp.lcp_index_build(torch.zeros((0, 8), dtype=torch.int16, device="cuda"), max_k=5,
                              capacity=40_000)
    allrows = []
    for t in range(30):
        r = g.step()
        allrows.append(r)
        lcp.lcp_index_insert(idx, dev(r))
        S = np.concatenate(allrows)
        if t < 5 or t % 10 == 9:
            ids, H = lcp.lcp_index_export(idx)
            w_ids, w_H = oracle.sorted_index(S)
            assert np.array_equal(ids.cpu().numpy(), w_ids), t
            assert np.array_equal(H.cpu().numpy(), w_H), t
            got = lcp.lcp_topk_batch(idx, dev(r), 5)
            want = oracle.topk_batch(S, r, 5)
            assert_same((got[0].cpu().numpy(), got[1].cpu().numpy()), want, "gnc step %d" % t)
    assert lcp.lcp_index_sync(idx) == 0
    # a large batch (radix path) and the capacity limit
    big = np.concatenate([g.step() for _ in range(3)])
    lcp.lcp_index_insert(idx, dev(big))
    S = np.concatenate(allrows + [big])
    ids, H = lcp.lcp_index_export(idx)
    w_ids, w_H = oracle.sorted_index(S)
    assert np.array_equal(ids.cpu().numpy(), w_ids) and np.array_equal(H.cpu().numpy(), w_H)
    with pytest.raises(lcp.LcpError) as e:
        lcp.lcp_index_insert(idx, dev(np.zeros((40_000, 8), np.uint16)))
    assert e.value.code == lcp.LCP_ERR_CAPACITY
    idx.close()


def test_determinism_alone_vs_batch_and_repeat(lcp):
    S, Qs, k = W.make_dataset("zipf500k_L32", N=100_000, Q=5_000)
    idx = lcp.lcp_index_build(dev(S), max_k=32)
    dq = dev(Qs)
    a = lcp.lcp_topk_batch(idx, dq, 32)
    b = lcp.lcp_topk_batch(idx, dq, 32)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    for i in (0, 17, 4999):
        one = lcp.lcp_topk_batch(idx, dq[i:i + 1].contiguous(), 32)
        assert torch.equal(one[0][0], a[0][i]) and torch.equal(one[1][0], a[1][i])
    # rebuilding gives the identical index
    idx2 = lcp.lcp_index_build(dev(S), max_k=32)
    e1, e2 = lcp.lcp_index_export(idx), lcp.lcp_index_export(idx2)
    assert torch.equal(e1[0], e2[0]) and torch.equal(e1[1], e2[1])
    idx.close()
    idx2.close()


def test_host_entry_points_match_device(lcp):
    S, Qs, k = W.make_dataset("tree16_u8", N=3000, Q=500)
    idx = lcp.lcp_index_build_host(host(S), max_k=k)
    hi, hl = lcp.lcp_topk_batch_host(idx, host(Qs), k)
    want = oracle.topk_batch(S, Qs, k)
    assert_same((hi.numpy(), hl.numpy()), want, "host entry points")
    # a batch large enough for the chunked, overlapped copy path
    Qb = np.tile(Qs, (1300, 1))  # 650,000 queries
    hi, hl = lcp.lcp_topk_batch_host(idx, host(Qb), k)
    di, dl = lcp.lcp_topk_batch(idx, dev(Qb), k)
    assert np.array_equal(hi.numpy(), di.cpu().numpy()) and np.array_equal(hl.numpy(), dl.cpu().numpy())
    assert np.array_equal(hi.numpy()[-500:], want[0]) and np.array_equal(hl.numpy()[-500:], want[1])
    idx.close()


def test_argument_errors(lcp):
    S = np.zeros((10, 4), np.uint8)
    idx = lcp.lcp_index_build(dev(S), max_k=8)
    with pytest.raises(lcp.LcpError) as e:
        lcp.lcp_topk_batch(idx, dev(S), 9)
    assert e.value.code == lcp.LCP_ERR_INVALID
    with pytest.raises(lcp.LcpError):
        lcp.lcp_index_insert(idx, dev(S))  # built without spare capacity
    idx.close()


def test_bounded_wait_reports_timeout_and_context_survives(lcp):
    assert lcp.lcp_debug_bounded_wait(1 << 14) == lcp.LCP_ERR_TIMEOUT
    S, Qs, k = W.make_dataset("tree16_u8", N=500, Q=50)
    assert_same(indexed(lcp, S, Qs, k), oracle.topk_batch(S, Qs, k), "after timeout")


def test_huge_tie_groups_take_the_exact_refinement(lcp):
    """Tie groups the on-device group sort does not take -- more than 2,048
    rows sharing packed word 0 (here 2,500), or a group of 33-2,048 rows in
    which a row shares word 1 with more than 64 others (here 700 rows equal
    on words 0 and 1) -- are ordered by the host-driven refinement after the
    graph build sees their count; the index and answers equal the oracle's."""
    rng = np.random.default_rng(12)
    N, L = 6_000, 24  # uint16: 4 tokens per word, so the first 8 tokens are words 0 and 1
    S = rng.integers(0, 50, size=(N, L)).astype(np.uint16)
    S[:2_500, :8] = 7          # one group of 2,500 rows tied on words 0-1
    S[2_500:3_200, :8] = 9     # and one of 700
    idx = lcp.lcp_index_build(dev(S), max_k=16)
    ids, H = lcp.lcp_index_export(idx)
    w_ids, w_H = oracle.sorted_index(S)
    assert np.array_equal(ids.cpu().numpy(), w_ids) and np.array_equal(H.cpu().numpy(), w_H)
    Qs = S[rng.integers(0, N, 200)].copy()
    Qs[::2, 10:] = 3
    got = lcp.lcp_topk_batch(idx, dev(Qs), 16)
    assert_same((got[0].cpu().numpy(), got[1].cpu().numpy()), oracle.topk_batch(S, Qs, 16), "huge groups")
    idx.close()
