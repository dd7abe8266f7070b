"""Streaming insert-then-query step replayed as a CUDA graph: every step's
answers equal the same step issued as direct calls on a twin index, the
graph is updated in place on most steps, and the index after the run equals
a fresh build of everything inserted (oracle)."""
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


def _empty(lcp, cap):
    return lcp.lcp_index_build(torch.zeros((0, 8), dtype=torch.int16, device="cuda"), max_k=5, capacity=cap)


def test_graph_step_equals_direct_calls(lcp):
    g = W.GncStream(sensors=1000, seed=5)
    steps = np.stack([g.step() for _ in range(260)])
    ds = dev(steps)
    a, b = _empty(lcp, 300_000), _empty(lcp, 300_000)
    step = lcp.Step(a, 1000, 1000, 5)
    for t in range(len(steps)):
        gi, gl = step.run(ds[t], ds[t])
        lcp.lcp_index_insert(b, ds[t])
        di, dl = lcp.lcp_topk_batch(b, ds[t], 5)
        assert torch.equal(gi, di) and torch.equal(gl, dl), t
        if t in (0, 1, 129, 259):
            S = steps[:t + 1].reshape(-1, 8)
            want = oracle.topk_batch(S, steps[t], 5)
            assert np.array_equal(gi.cpu().numpy(), want[0]) and np.array_equal(gl.cpu().numpy(), want[1]), t
    runs, inst = step.stats()
    assert runs == len(steps)
    # N grows from 1,000 to 260,000: the graph is re-instantiated only when
    # the number of kernels changes (min-tree and sparse-table levels)
    assert 1 <= inst <= 16, inst
    ids, H = lcp.lcp_index_export(a)
    w_ids, w_H = oracle.sorted_index(steps.reshape(-1, 8))
    assert np.array_equal(ids.cpu().numpy(), w_ids) and np.array_equal(H.cpu().numpy(), w_H)
    assert lcp.lcp_index_sync(a) == 0
    step.close()
    a.close()
    b.close()


def test_graph_step_insert_only_query_only_and_capacity(lcp):
    g = W.GncStream(sensors=500, seed=7)
    r0, r1 = g.step(), g.step()
    a = _empty(lcp, 1_000)
    ins = lcp.Step(a, 500, 0, 5)
    qry = lcp.Step(a, 0, 500, 3)
    ins.run(dev(r0), dev(r0[:0]))
    gi, gl = qry.run(dev(r0[:0]), dev(r1))
    want = oracle.topk_batch(r0, r1, 3)
    assert np.array_equal(gi.cpu().numpy(), want[0]) and np.array_equal(gl.cpu().numpy(), want[1])
    ins.run(dev(r1), dev(r1[:0]))
    assert a.N == 1_000
    with pytest.raises(lcp.LcpError) as e:  # full: the index is left as it was
        ins.run(dev(r1), dev(r1[:0]))
    assert e.value.code == lcp.LCP_ERR_CAPACITY
    gi, gl = qry.run(dev(r0[:0]), dev(r1))
    want = oracle.topk_batch(np.concatenate([r0, r1]), r1, 3)
    assert np.array_equal(gi.cpu().numpy(), want[0]) and np.array_equal(gl.cpu().numpy(), want[1])
    with pytest.raises(lcp.LcpError):
        lcp.Step(a, 5_000, 10, 5)  # more rows than the graph-capturable insert takes
    with pytest.raises(lcp.LcpError):
        lcp.Step(a, 10, 10, 6)     # k above the index's max_k
    ins.close()
    qry.close()
    a.close()
