"""Sharded layout on one GPU: P shard indexes over id ranges, their answers
merged by lcp_shard_merge, equal byte for byte to one index over all rows."""
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


def _sharded(lcp, S, Qs, k, P):
    from paper_2602_04936_b300.shard import shard_bounds
    bases, counts = shard_bounds(len(S), P)
    dq = dev(Qs)
    parts = []
    for b, c in zip(bases, counts):
        ix = lcp.lcp_index_build(dev(S[b:b + c]), max_k=k)
        parts.append(lcp.lcp_topk_batch(ix, dq, k))
        ix.close()
    ids = torch.stack([p[0] for p in parts])
    lc = torch.stack([p[1] for p in parts])
    return lcp.lcp_shard_merge(ids, lc, bases)


@pytest.mark.parametrize("P", [1, 2, 3, 7])
def test_shard_merge_equals_single_index(lcp, P):
    S, Qs, k = W.make_dataset("zipf500k_L32", N=60_000, Q=3_000)
    got = _sharded(lcp, S, Qs, k, P)
    one = lcp.lcp_index_build(dev(S), max_k=k)
    want = lcp.lcp_topk_batch(one, dev(Qs), k)
    assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])
    w_ids, w_lcp = oracle.topk_batch(S, Qs[:200], k)
    assert np.array_equal(got[0][:200].cpu().numpy(), w_ids) and np.array_equal(got[1][:200].cpu().numpy(), w_lcp)
    one.close()


def test_shard_merge_padding_and_tiny_shards(lcp):
    # 5 shards of 3-4 rows and k = 20 > N: every answer ends in padding
    S, Qs, _ = W.make_dataset("tree16_u8", N=17, Q=40)
    got = _sharded(lcp, S, Qs, 20, 5)
    w_ids, w_lcp = oracle.topk_batch(S, Qs, 20)
    assert np.array_equal(got[0].cpu().numpy(), w_ids) and np.array_equal(got[1].cpu().numpy(), w_lcp)


def test_sharded_index_single_process(lcp):
    from paper_2602_04936_b300.shard import ShardedIndex
    S, Qs, k = W.make_dataset("tree16_u8", N=2_000, Q=300)
    sh = ShardedIndex(dev(S), len(S), max_k=k)
    ids, lc = sh.topk(dev(Qs), k)
    w_ids, w_lcp = oracle.topk_batch(S, Qs, k)
    assert np.array_equal(ids.cpu().numpy(), w_ids) and np.array_equal(lc.cpu().numpy(), w_lcp)


def test_shard_merge_argument_errors(lcp):
    z = torch.zeros((2, 4, 3), dtype=torch.int32, device="cuda")
    zl = torch.zeros((2, 4, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        lcp.lcp_shard_merge(z, zl, [0])
    with pytest.raises(lcp.LcpError):
        lcp.lcp_shard_merge(z, zl, [0, -5])
