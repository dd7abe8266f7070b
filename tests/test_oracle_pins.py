"""Pins for the CPU oracle: each test checks it against something other than
itself -- a hand-worked example, exhaustive enumeration with Python's own
sort and os.path.commonprefix, the literal pointer trie of Algorithms 1-4,
the ultrametric property (Theorem 1) and the descent lemma (App. A).

A plausible mistake in the oracle (a dropped tie-break, a reversed order, an
off-by-one LCP, a wrong pad, an unstable sort) fails at least one of these.
"""
import itertools
import os
import random

import numpy as np
import pytest

import oracle
import trie_checker as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_example.txt")


def _parse_golden():
    S, cases, sorted_case = [], [], None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, rest = line.split(" ", 1)
            if tag == "S":
                S.append([int(x) for x in rest.split()])
            elif tag == "Q":
                q, k, ids, lcps = [p.strip() for p in rest.split("|")]
                cases.append(([int(x) for x in q.split()], int(k),
                              [int(x) for x in ids.split()], [int(x) for x in lcps.split()]))
            elif tag == "SORTED":
                ids, H = [p.strip() for p in rest.split("|")]
                sorted_case = ([int(x) for x in ids.split()], [int(x) for x in H.split()])
    return np.array(S, np.uint8), cases, sorted_case


def _brute(S, q, k):
    """Independent route: os.path.commonprefix + Python's sorted()."""
    lc = [len(os.path.commonprefix([tuple(int(x) for x in s), tuple(int(x) for x in q)]))
          for s in S]
    order = sorted(range(len(S)), key=lambda i: (-lc[i], i))[:k]
    ids = order + [-1] * (k - len(order))
    lcs = [lc[i] for i in order] + [0] * (k - len(order))
    return ids, lcs


def test_hand_example_topk():
    S, cases, _ = _parse_golden()
    for q, k, ids, lcps in cases:
        got_ids, got_lcp = oracle.topk(S, np.array(q, np.uint8), k)
        assert got_ids.tolist() == ids, (q, k)
        assert got_lcp.tolist() == lcps, (q, k)


def test_hand_example_sorted_index():
    S, _, (ids, H) = _parse_golden()
    got_ids, got_H = oracle.sorted_index(S)
    assert got_ids.tolist() == ids
    assert got_H.tolist() == H


def test_hand_example_batch_matches_single():
    S, cases, _ = _parse_golden()
    Qs = np.array([c[0] for c in cases], np.uint8)
    ids, lc = oracle.topk_batch(S, Qs, 9, threads=3)
    for r, (q, _, _, _) in enumerate(cases):
        i1, l1 = oracle.topk(S, np.array(q, np.uint8), 9)
        assert ids[r].tolist() == i1.tolist() and lc[r].tolist() == l1.tolist()


@pytest.mark.parametrize("sigma,L", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_exhaustive_small_alphabets(sigma, L):
    """Every query in Sigma^L, random multisets N <= 12, every k in 1..N+2."""
    rng = random.Random(sigma * 100 + L)
    all_q = list(itertools.product(range(sigma), repeat=L))
    for trial in range(6):
        N = rng.randint(0, 12)
        S = np.array([[rng.randrange(sigma) for _ in range(L)] for _ in range(N)],
                     np.uint8).reshape(N, L)
        root = T.build(S)
        for q in all_q:
            qa = np.array(q, np.uint8)
            for k in range(1, N + 3):
                got_ids, got_lcp = oracle.topk(S, qa, k)
                b_ids, b_lcp = _brute(S, q, k)
                t_ids, t_lcp = T.topk_by_trie(root, q, k, N)
                assert got_ids.tolist() == b_ids == t_ids, (S.tolist(), q, k)
                assert got_lcp.tolist() == b_lcp == t_lcp, (S.tolist(), q, k)


def test_uint16_tokens_high_values():
    """Unsigned order and LCP with tokens near 0xFFFF (uint16)."""
    S = np.array([[0xFFFF, 1, 2], [0xFFFF, 1, 3], [0x7FFF, 1, 2], [0, 0, 0], [0xFFFF, 1, 2]],
                 np.uint16)
    q = np.array([0xFFFF, 1, 2], np.uint16)
    ids, lc = oracle.topk(S, q, 5)
    assert ids.tolist() == [0, 4, 1, 2, 3]
    assert lc.tolist() == [3, 3, 2, 0, 0]
    sid, H = oracle.sorted_index(S)
    assert sid.tolist() == [3, 2, 0, 4, 1]
    assert H.tolist() == [0, 0, 0, 3, 2]


def test_lcp_invariants_and_ultrametric():
    """LCP(q,q)=L, symmetry, and Theorem 1: LCP(s,u) >= min(LCP(s,t), LCP(t,u))."""
    rng = np.random.default_rng(7)
    for L, tb in ((1, 1), (5, 1), (9, 2), (33, 2)):
        dt = np.uint8 if tb == 1 else np.uint16
        X = rng.integers(0, 3, size=(60, L)).astype(dt)
        for _ in range(300):
            a, b, c = X[rng.integers(0, 60, 3)]
            assert oracle.lcp(a, a) == L
            assert oracle.lcp(a, b) == oracle.lcp(b, a)
            assert oracle.lcp(a, c) >= min(oracle.lcp(a, b), oracle.lcp(b, c))


def _random_prefixy(rng, N, L, sigma, dt):
    """Rows sharing prefixes: random walks down a small random tree."""
    base = rng.integers(0, sigma, size=(max(N // 4, 1), L))
    rows = base[rng.integers(0, base.shape[0], N)].copy()
    cut = rng.integers(0, L + 1, N)
    for i in range(N):
        rows[i, cut[i]:] = rng.integers(0, sigma, L - cut[i])
    return rows.astype(dt)


@pytest.mark.parametrize("L,tb,sigma", [(4, 1, 3), (7, 1, 4), (12, 2, 5), (3, 2, 70000 // 2)])
def test_sorted_index_against_python_sort(L, tb, sigma):
    rng = np.random.default_rng(L * 13 + tb)
    dt = np.uint8 if tb == 1 else np.uint16
    sigma = min(sigma, 256 if tb == 1 else 65536)
    S = _random_prefixy(rng, 500, L, sigma, dt)
    ids, H = oracle.sorted_index(S)
    expect = sorted(range(len(S)), key=lambda i: (tuple(int(x) for x in S[i]), i))
    assert ids.tolist() == expect
    for p in range(len(S)):
        if p == 0:
            assert H[p] == 0
        else:
            cp = os.path.commonprefix([tuple(S[ids[p - 1]].tolist()), tuple(S[ids[p]].tolist())])
            assert H[p] == len(cp)


def test_sorted_order_invariants():
    """Contiguity of {p : LCP(q, row p) >= d}; range-min of H equals range LCP;
    and the count with LCP >= d equals the trie subtree size on q's path
    (Algorithm 2)."""
    rng = np.random.default_rng(3)
    L = 6
    S = _random_prefixy(rng, 300, L, 3, np.uint8)
    ids, H = oracle.sorted_index(S)
    rows = S[ids]
    root = T.build(S)
    # range minimum of H over (i, j] equals LCP(row i, row j)
    for _ in range(400):
        i, j = sorted(rng.integers(0, len(S), 2))
        if i == j:
            continue
        assert H[i + 1:j + 1].min() == oracle.lcp(rows[i], rows[j])
    for _ in range(100):
        q = rng.integers(0, 3, L).astype(np.uint8)
        lam = np.array([oracle.lcp(q, r) for r in rows])
        path = T.descend(root, q)
        for d in range(L + 1):
            where = np.nonzero(lam >= d)[0]
            if len(where):
                assert where[-1] - where[0] + 1 == len(where)  # contiguous
            if d < len(path):
                assert len(where) == path[d].size  # Algorithm 2 subtree size
            else:
                assert len(where) == 0


def test_descent_lemma_and_bfs_lcp_column():
    """App. A: after descending to depth d, items outside T_v have LCP < d
    (strict).  When |T_v| >= k, the LCP column of literal Algorithm 4 (BFS
    order) equals the oracle's LCP column."""
    rng = np.random.default_rng(11)
    L = 5
    S = _random_prefixy(rng, 200, L, 3, np.uint8)
    root = T.build(S)
    checked = 0
    for _ in range(300):
        q = rng.integers(0, 3, L).astype(np.uint8)
        path = T.descend(root, q)
        v, d = path[-1], len(path) - 1
        inside = set(T.items_in(v))
        for i in range(len(S)):
            if i not in inside:
                assert oracle.lcp(q, S[i]) < d
        k = int(rng.integers(1, 12))
        if v.size >= k:
            bfs = T.collect_bfs(v, k)
            _, o_lcp = oracle.topk(S, q, k)
            assert [oracle.lcp(q, S[i]) for i in bfs] == o_lcp.tolist()
            checked += 1
    assert checked > 20


def test_k1_member_query():
    """k=1 with q in S returns (smallest id holding q, L) -- the distinguishing
    query of the space lower bound's argument (Sec. 4.1)."""
    rng = np.random.default_rng(5)
    S = rng.integers(0, 2, size=(64, 6)).astype(np.uint8)
    for i in range(64):
        ids, lc = oracle.topk(S, S[i], 1)
        first = min(j for j in range(64) if (S[j] == S[i]).all())
        assert ids[0] == first and lc[0] == 6


def test_empty_and_degenerate():
    S = np.zeros((0, 3), np.uint8)
    ids, lc = oracle.topk(S, np.array([1, 2, 3], np.uint8), 4)
    assert ids.tolist() == [-1] * 4 and lc.tolist() == [0] * 4
    S = np.ones((5, 3), np.uint8)  # all identical
    ids, lc = oracle.topk(S, np.array([1, 1, 1], np.uint8), 3)
    assert ids.tolist() == [0, 1, 2] and lc.tolist() == [3, 3, 3]
    ids, lc = oracle.topk(S, np.array([1, 1, 2], np.uint8), 7)
    assert ids.tolist() == [0, 1, 2, 3, 4, -1, -1] and lc.tolist() == [2] * 5 + [0, 0]
    with pytest.raises(ValueError):
        oracle.topk(S, np.array([1, 1, 1], np.uint8), 0)


def test_workload_generators_are_deterministic_and_shaped():
    """Inputs are seeded: regenerating gives identical bytes; shapes match."""
    import workloads as W
    a = W.make_dataset("tree16_u8", N=500, Q=50)
    b = W.make_dataset("tree16_u8", N=500, Q=50)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all() and a[2] == 10
    assert a[0].dtype == np.uint8 and a[0].max() < 16
    # 4-ary tree over the first 8 positions: at most 4 children per prefix
    S = a[0]
    for d in range(8):
        kids = {}
        for r in S:
            kids.setdefault(tuple(r[:d]), set()).add(int(r[d]))
        assert max(len(v) for v in kids.values()) <= 4
    z = W.make_dataset("zipf500k_L32", N=2000, Q=100)
    assert z[0].dtype == np.uint16 and z[0].shape == (2000, 32) and z[0].max() < 1024
    g = W.GncStream(sensors=10, seed=5)
    r0 = g.step()
    assert r0.shape == (10, 8) and r0[:, 2:].max() <= 9
    # uniform rows (TAL shape): deterministic, chunking-independent, every
    # first-token bucket near n / 256
    u = W.uniform_rows(51_200, 16, 256, 6)
    assert np.array_equal(u, W.uniform_rows(51_200, 16, 256, 6, chunk=777))
    counts = np.bincount(u[:, 0], minlength=256)
    assert u.dtype == np.uint8 and counts.min() > 120 and counts.max() < 290
    assert W.uniform_rows(10, 4, 1000, 1).dtype == np.uint16


def test_zipf_generator_c_path_matches_numpy_reference():
    """workloads/gen.c draws exactly what the numpy definition draws."""
    import workloads as W
    for N, L, V, s in [(1500, 32, 1024, 1.1), (800, 64, 32768, 1.05), (300, 8, 16, 1.0)]:
        a = W.zipf_prefix_rows(N, L, V, s, 7, impl="c")
        b = W.zipf_prefix_rows(N, L, V, s, 7, impl="numpy")
        assert np.array_equal(a, b)
        qa = W.zipf_prefix_queries(a, 400, V, s, 7, impl="c")
        qb = W.zipf_prefix_queries(a, 400, V, s, 7, impl="numpy")
        assert np.array_equal(qa, qb)


@pytest.mark.parametrize("sigma,L", [(2, 3), (3, 3), (2, 4)])
def test_bfs_and_tal_against_pointer_trie(sigma, L):
    """The BFS-order variant (Algorithms 3 + 4) and the TAL bucket scan against
    the pointer trie, every query in Sigma^L, random multisets N <= 12."""
    rng = random.Random(sigma * 1000 + L)
    all_q = np.array(list(itertools.product(range(sigma), repeat=L)), np.uint8).reshape(-1, L)
    for trial in range(5):
        N = rng.randint(0, 12)
        S = np.array([[rng.randrange(sigma) for _ in range(L)] for _ in range(N)],
                     np.uint8).reshape(N, L)
        root = T.build(S)
        for k in (1, 2, 5, 14):
            b_ids, b_lcp = oracle.topk_bfs(S, all_q, k)
            for qi, q in enumerate(all_q):
                t_ids, t_lcp = T.query_bfs(root, q, k)
                assert b_ids[qi].tolist() == t_ids and b_lcp[qi].tolist() == t_lcp, (S.tolist(), q, k)
            for d in range(L + 1):
                a_ids, a_lcp = oracle.tal_topk(S, all_q, k, d)
                for qi, q in enumerate(all_q):
                    t_ids, t_lcp = T.tal_by_trie(root, q, k, d)
                    assert a_ids[qi].tolist() == t_ids and a_lcp[qi].tolist() == t_lcp, (S.tolist(), q, k, d)


def test_bfs_and_tal_reduce_to_the_definition():
    """TAL at depth 0 scans everything, so it is the Definition's top k; a
    bucket holding >= k items gives the Definition's answer too (every item
    outside has a smaller LCP).  BFS order differs from the Definition only in
    which ties it keeps: its LCP column equals the Definition's when |T_v| >= k."""
    S, Qs, _ = __import__("workloads").make_dataset("tree16_u8", N=600, Q=80)
    k = 7
    want_i, want_l = oracle.topk_batch(S, Qs, k)
    t_i, t_l = oracle.tal_topk(S, Qs, k, 0)
    assert np.array_equal(t_i, want_i) and np.array_equal(t_l, want_l)
    for d in (1, 2, 3):
        t_i, t_l = oracle.tal_topk(S, Qs, k, d)
        full = (t_i >= 0).all(axis=1)
        assert full.any() and np.array_equal(t_i[full], want_i[full]) and np.array_equal(t_l[full], want_l[full])
    b_i, b_l = oracle.topk_bfs(S, Qs, k)
    full = (b_i >= 0).all(axis=1)
    assert full.any() and np.array_equal(b_l[full], want_l[full])



# ---- rows longer than 255 tokens: 16-bit LCPs (the paper's sustained shape) ----

def _long_rows(rng, N, L, sigma, dt):
    """Rows sharing long prefixes, exact duplicates, and rows that differ from
    another only in the last token (LCP L - 1 against L)."""
    base = rng.integers(0, sigma, size=(max(N // 4, 1), L))
    rows = base[rng.integers(0, base.shape[0], N)].copy()
    cut = rng.integers(L - 40, L + 1, N)
    for i in range(N):
        if cut[i] < L:
            rows[i, cut[i]:] = rng.integers(0, sigma, L - cut[i])
    rows[N // 2, -1] = (rows[N // 2, -1] + 1) % sigma  # last-token neighbour of a base row
    rows[N - 1] = rows[0]  # an exact duplicate
    return rows.astype(dt)


@pytest.mark.parametrize("L,tb,sigma", [(256, 2, 3), (300, 1, 2), (256, 1, 4), (1000, 2, 2)])
def test_wide_topk_against_python(L, tb, sigma):
    """topk_wide against os.path.commonprefix + sorted() at L >= 256, where an
    LCP of L needs more than 8 bits; queries include exact members, members
    with only the last token changed, and random rows."""
    rng = np.random.default_rng(L + tb)
    dt = np.uint8 if tb == 1 else np.uint16
    S = _long_rows(rng, 40, L, sigma, dt)
    Qs = np.concatenate([S[rng.integers(0, 40, 6)], S[rng.integers(0, 40, 6)], rng.integers(0, sigma, (4, L))])
    Qs[6:12, -1] = (Qs[6:12, -1].astype(np.int64) + 1) % sigma
    Qs = Qs.astype(dt)
    for k in (1, 3, 45):
        ids, lc = oracle.topk_wide(S, Qs, k, threads=2)
        assert lc.dtype == np.uint16
        for r in range(len(Qs)):
            w_ids, w_lc = _brute(S, Qs[r], k)
            assert ids[r].tolist() == w_ids and lc[r].tolist() == w_lc, (k, r)
    # a member query's top-1 is its smallest equal row, with LCP L (> 255)
    ids, lc = oracle.topk_wide(S, S[:1], 1)
    eq = np.nonzero((S == S[0]).all(1))[0]
    assert ids[0, 0] == eq.min() and lc[0, 0] == L


def test_wide_topk_equals_narrow_below_256():
    """For L <= 255 both oracles state the same definition: equal outputs."""
    rng = np.random.default_rng(5)
    for L, tb, sigma in ((16, 1, 3), (255, 2, 2), (33, 2, 5)):
        dt = np.uint8 if tb == 1 else np.uint16
        S = _random_prefixy(rng, 300, L, sigma, dt)
        Qs = S[rng.integers(0, 300, 50)].copy()
        Qs[::2, L // 2:] = rng.integers(0, sigma, (25, L - L // 2))
        a = oracle.topk_batch(S, Qs, 20)
        b = oracle.topk_wide(S, Qs, 20)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].astype(np.uint16), b[1])


def test_wide_sorted_index_against_python_sort():
    rng = np.random.default_rng(9)
    S = _long_rows(rng, 60, 257, 3, np.uint16)
    ids, H = oracle.sorted_index_wide(S)
    want = sorted(range(len(S)), key=lambda i: (tuple(int(x) for x in S[i]), i))
    assert ids.tolist() == want
    for p in range(1, len(S)):
        a, b = S[want[p - 1]], S[want[p]]
        assert H[p] == len(os.path.commonprefix([tuple(a.tolist()), tuple(b.tolist())]))
    assert H.max() == 257  # duplicates present: an LCP that needs 16 bits
