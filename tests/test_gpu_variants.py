"""The paper's own query modes on the GPU against the oracle: BFS order
(Algorithms 3 + 4 as printed) and the TAL bucket scan."""
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


def _same(got, want, what):
    gi, gl = got[0].cpu().numpy(), got[1].cpu().numpy()
    bad = np.where((gi != want[0]).any(1) | (gl != want[1]).any(1))[0]
    assert len(bad) == 0, "%s: %d rows differ, first %d: got %s / %s want %s / %s" % (
        what, len(bad), bad[0], gi[bad[0]], gl[bad[0]], want[0][bad[0]], want[1][bad[0]])


CASES = [("tree16_u8", 3_000, 400), ("zipf500k_L32", 40_000, 200)]


@pytest.mark.parametrize("name,N,Q", CASES)
def test_bfs_matches_oracle(lcp, name, N, Q):
    S, Qs, _ = W.make_dataset(name, N=N, Q=Q)
    idx = lcp.lcp_index_build(dev(S), max_k=32)
    for k in (1, 10, 100, 1000):
        _same(lcp.lcp_topk_bfs(idx, dev(Qs), k), oracle.topk_bfs(S, Qs, k), "%s bfs k=%d" % (name, k))
    idx.close()


@pytest.mark.parametrize("name,N,Q", CASES)
def test_tal_matches_oracle(lcp, name, N, Q):
    S, Qs, _ = W.make_dataset(name, N=N, Q=Q)
    L = S.shape[1]
    idx = lcp.lcp_index_build(dev(S), max_k=32)
    for d in (0, 1, 2, 3, L):
        for k in (1, 10, 32):
            _same(lcp.lcp_tal_topk(idx, dev(Qs[:60] if d == 0 else Qs), k, d),
                  oracle.tal_topk(S, Qs[:60] if d == 0 else Qs, k, d), "%s tal d=%d k=%d" % (name, d, k))
    idx.close()


def test_modes_small_and_degenerate(lcp):
    S = np.array([[1, 2, 3], [1, 2, 4], [1, 3, 0], [1, 2, 3], [2, 0, 0]], np.uint8)
    Qs = np.array([[1, 2, 9], [3, 3, 3], [1, 2, 3], [2, 0, 0]], np.uint8)
    idx = lcp.lcp_index_build(dev(S), max_k=8)
    for k in (1, 3, 7):
        _same(lcp.lcp_topk_bfs(idx, dev(Qs), k), oracle.topk_bfs(S, Qs, k), "bfs k=%d" % k)
        for d in range(4):
            _same(lcp.lcp_tal_topk(idx, dev(Qs), k, d), oracle.tal_topk(S, Qs, k, d), "tal d=%d" % d)
    with pytest.raises(lcp.LcpError):
        lcp.lcp_tal_topk(idx, dev(Qs), 33, 1)
    with pytest.raises(lcp.LcpError):
        lcp.lcp_tal_topk(idx, dev(Qs), 5, 4)
    idx.close()


def test_tal_workload_sampled(lcp):
    """The TAL shape: uniform first tokens over 256 values, depth 1 (256
    buckets), here at N = 2M; sampled queries against the oracle."""
    N, L = 2_000_000, 16
    S = W.uniform_rows(N, L, 256, 11)
    Qs = W.uniform_rows(512, L, 256, 12)
    idx = lcp.lcp_index_build(dev(S), max_k=32)
    got = lcp.lcp_tal_topk(idx, dev(Qs), 10, 1)
    sel = np.arange(0, 512, 64)
    want = oracle.tal_topk(S, Qs[sel], 10, 1)
    _same((got[0][sel], got[1][sel]), want, "tal 2M sampled")
    # a full bucket (>= k rows) ranks like the Definition
    dq = lcp.lcp_topk_batch(idx, dev(Qs), 10)
    assert torch.equal(dq[0], got[0]) and torch.equal(dq[1], got[1])
    idx.close()
