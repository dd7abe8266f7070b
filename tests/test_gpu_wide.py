"""Top-1 with 16-bit LCPs over rows longer than 255 tokens (the paper's
sustained benchmark shape, Sec. 7 Table 4 and App. C: top-1, max_len 256)
against the CPU oracle's Definition "Top-k LCP Retrieval" with k = 1.

The edge the 16-bit LCP exists for: a query equal to a stored row (LCP = L,
e.g. 256) next to rows that differ from it only in the last token (LCP
L - 1); the smallest id among the exact copies must win, with LCP L.
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


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a).cuda()


def _long_rows(rng, N, L, sigma, dt):
    base = rng.integers(0, sigma, size=(max(N // 8, 1), L))
    rows = base[rng.integers(0, base.shape[0], N)].copy()
    cut = rng.integers(0, L + 1, N)
    cut[::3] = L - 1 - rng.integers(0, 3, len(cut[::3]))  # deep shared prefixes
    for i in range(N):
        if cut[i] < L:
            rows[i, cut[i]:] = rng.integers(0, sigma, L - cut[i])
    rows[-50:] = rows[:50]                     # exact duplicates (later ids)
    rows[-100:-50] = rows[:50]
    rows[-100:-50, -1] = (rows[-100:-50, -1] + 1) % sigma  # last-token neighbours
    return rows.astype(dt)


def _queries(rng, S, Q, sigma):
    N, L = S.shape
    Qs = S[rng.integers(0, N, Q)].copy()
    n = Q // 4
    Qs[n:2 * n, -1] = (Qs[n:2 * n, -1].astype(np.int64) + 1) % sigma       # last token changed
    Qs[2 * n:3 * n, L // 2:] = rng.integers(0, sigma, (n, L - L // 2))      # half the row
    Qs[3 * n:] = rng.integers(0, sigma, (Q - 3 * n, L))                     # random
    Qs[0] = 0
    Qs[1] = np.iinfo(S.dtype).max
    return Qs.astype(S.dtype)


def _check(got, want, what):
    gi, gl = got[0].cpu().numpy(), got[1].cpu().numpy().view(np.uint16)
    wi, wl = want[0][:, 0], want[1][:, 0]
    bad = np.nonzero((gi != wi) | (gl != wl))[0]
    assert len(bad) == 0, "%s: %d/%d differ; first q=%d got (%d, %d) want (%d, %d)" % (
        what, len(bad), len(gi), bad[0], gi[bad[0]], gl[bad[0]], wi[bad[0]], wl[bad[0]])


@pytest.mark.parametrize("N,L,tb,sigma", [(3000, 256, 2, 3), (5000, 256, 1, 2), (2000, 300, 1, 4),
                                          (1500, 1024, 2, 2), (700, 257, 2, 50), (1, 256, 2, 2),
                                          (40000, 256, 1, 3)])
def test_wide_index_and_scan_match_oracle(lcp, N, L, tb, sigma):
    rng = np.random.default_rng(N + L + tb)
    dt = np.uint8 if tb == 1 else np.uint16
    S = _long_rows(rng, N, L, sigma, dt) if N >= 200 else rng.integers(0, sigma, (N, L)).astype(dt)
    Qs = _queries(rng, S, 400, sigma)
    want = oracle.topk_wide(S, Qs, 1)
    idx = lcp.lcp_index_build(dev(S), max_k=1)
    ids, _ = lcp.lcp_index_export(idx)
    assert np.array_equal(ids.cpu().numpy(), oracle.sorted_index_wide(S)[0])
    got = lcp.lcp_top1_wide(idx, dev(Qs))
    torch.cuda.synchronize()
    assert lcp.lcp_index_sync(idx) == 0
    _check(got, want, "indexed top-1")
    _check(lcp.lcp_scan_top1_wide(dev(S), dev(Qs)), want, "full-scan top-1")
    if N >= 200:
        assert want[1].max() == L  # exact copies were queried: LCP L > 255
    idx.close()


@pytest.mark.parametrize("N,L,tb,sigma", [(1000, 16, 1, 16), (20000, 8, 1, 2), (5000, 33, 2, 4),
                                          (3000, 255, 1, 2)])
def test_top1_wide_on_narrow_indexes(lcp, N, L, tb, sigma):
    """lcp_top1_wide serves any index: on rows of <= 255 tokens it equals the
    8-bit path's top-1 and the oracle."""
    rng = np.random.default_rng(N * 3 + L)
    dt = np.uint8 if tb == 1 else np.uint16
    S = _long_rows(rng, N, L, sigma, dt)
    Qs = _queries(rng, S, 500, sigma)
    want = oracle.topk_wide(S, Qs, 1)
    idx = lcp.lcp_index_build(dev(S), max_k=8)
    got = lcp.lcp_top1_wide(idx, dev(Qs))
    eight = lcp.lcp_topk_batch(idx, dev(Qs), 1)
    torch.cuda.synchronize()
    _check(got, want, "wide top-1 on a narrow index")
    assert torch.equal(eight[0][:, 0], got[0]) and torch.equal(eight[1][:, 0].to(torch.int16), got[1])
    _check(lcp.lcp_scan_top1_wide(dev(S), dev(Qs)), want, "full-scan top-1, narrow rows")
    idx.close()


def test_sustained_shape_full_size(lcp):
    """The sustained shape at full size: 2M rows of 256 uint16 tokens; 1,000
    of its queries against the oracle, 100,000 indexed answers against the
    full scan, and single-query calls equal to the batch."""
    S, Qs, k = W.make_dataset("sustained2m_L256")
    assert S.shape == (2_000_000, 256) and k == 1
    dS = dev(S)
    idx = lcp.lcp_index_build(dS, max_k=1)
    dq = dev(Qs)
    got = lcp.lcp_top1_wide(idx, dq)
    pick = np.sort(np.random.default_rng(7).choice(len(Qs), 1000, replace=False))
    sc = lcp.lcp_scan_top1_wide(dS, dq[torch.from_numpy(pick).cuda()])
    torch.cuda.synchronize()
    assert lcp.lcp_index_sync(idx) == 0
    want = oracle.topk_wide(S, Qs[pick], 1)
    _check((got[0][torch.from_numpy(pick).cuda()], got[1][torch.from_numpy(pick).cuda()]), want,
           "sustained indexed vs oracle")
    _check(sc, want, "sustained full scan vs oracle")
    for i in pick[:20]:
        one = lcp.lcp_top1_wide(idx, dq[i:i + 1])
        assert int(one[0][0]) == int(got[0][i]) and int(one[1][0]) == int(got[1][i])
    # copies keep 128 tokens of a stored row: their best LCP is at least 128
    copies = (want[1][:, 0] >= 128).mean()
    assert copies > 0.4
    idx.close()


def test_wide_index_argument_errors(lcp):
    S = np.zeros((100, 256), np.uint16)
    with pytest.raises(lcp.LcpError) as e:  # rows longer than 255 tokens: top-1 only
        lcp.lcp_index_build(dev(S), max_k=2)
    assert e.value.code == lcp.LCP_ERR_INVALID
    with pytest.raises(lcp.LcpError):
        lcp.lcp_index_build(dev(S), max_k=1, capacity=200)  # no inserts into a wide index
    with pytest.raises(lcp.LcpError):
        lcp.lcp_index_build(dev(np.zeros((10, 1025), np.uint16)), max_k=1)  # beyond LCP_MAX_L_WIDE
    idx = lcp.lcp_index_build(dev(S), max_k=1)
    with pytest.raises(lcp.LcpError) as e:
        lcp.lcp_topk_batch(idx, dev(S[:3]), 1)  # an 8-bit LCP cannot hold 256
    assert e.value.code == lcp.LCP_ERR_INVALID
    ids, H = lcp.lcp_index_export(idx)
    assert H is None and ids.numel() == 100
    got = lcp.lcp_top1_wide(idx, dev(S[:3]))
    assert got[0].tolist() == [0, 0, 0] and got[1].tolist() == [256, 256, 256]
    idx.close()
