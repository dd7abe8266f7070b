"""Autotuned launch shapes change the schedule only: every shape returns the
same bytes, and the tuner installs one of them for the batch's class."""
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


def test_every_shape_same_answer_and_tuner(lcp):
    S, Qs, k = W.make_dataset("zipf500k_L32", N=100_000, Q=20_000)
    idx = lcp.lcp_index_build(dev(S), max_k=k)
    dq = dev(Qs)
    base = lcp.lcp_topk_batch(idx, dq, k)
    w_ids, w_lcp = oracle.topk_batch(S, Qs[:300], k)
    assert np.array_equal(base[0][:300].cpu().numpy(), w_ids) and np.array_equal(base[1][:300].cpu().numpy(), w_lcp)
    for lw in (0, 1, 2):  # lane, warp, lane over the staged top levels
        for qpw in (0, 1, 2, 4, 8, 16, 32):  # 0: the fused kernel
            lcp.lcp_set_search_shape(idx, len(Qs), k, qpw, lw)
            got = lcp.lcp_topk_batch(idx, dq, k)
            assert torch.equal(got[0], base[0]) and torch.equal(got[1], base[1]), (qpw, lw)
    r = lcp.lcp_autotune(idx, dq, k)
    assert r["qpw"] in (0, 1, 2, 4, 8, 16, 32) and r["locate_warp"] in (0, 1, 2)
    assert 0 < r["best_ms"] <= r["default_ms"] * 1.0001
    got = lcp.lcp_topk_batch(idx, dq, k)
    assert torch.equal(got[0], base[0]) and torch.equal(got[1], base[1])
    with pytest.raises(lcp.LcpError):
        lcp.lcp_set_search_shape(idx, len(Qs), k, 64, 0)
    with pytest.raises(lcp.LcpError):
        lcp.lcp_set_search_shape(idx, len(Qs), k, 4, 3)
    idx.close()
