"""Serving session on the GPU: requests against several resident indexes,
admitted under a memory budget and overlapped on several streams; every
result equals the same request served alone (lcp_topk_batch) and the oracle."""
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


def _dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a).cuda()


def _pinned(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a).pin_memory()


def test_session_mix_equals_alone(lcp):
    rng = np.random.default_rng(4)
    specs = [(3_000, 16, 1024, 1.1), (50_000, 32, 32768, 1.05), (200_000, 64, 32768, 1.05)]
    data, idxs = [], []
    for i, (N, L, V, s) in enumerate(specs):
        S = W.zipf_prefix_rows(N, L, V, s, 40 + i)
        Qs = W.zipf_prefix_queries(S, 6_000, V, s, 40 + i)
        data.append((S, Qs))
        idxs.append(lcp.lcp_index_build(_dev(S), max_k=100))
    sess = lcp.Session(mem_budget=8 << 20, max_inflight=6, streams=4)
    slots = [sess.add_index(ix) for ix in idxs]
    reqs = []
    for r in range(60):
        j = int(rng.integers(0, 3))
        Q = int(np.exp(rng.uniform(0, np.log(2000))))
        k = int(rng.choice([1, 10, 100]))
        off = int(rng.integers(0, 6_000 - Q))
        q = data[j][1][off:off + Q]
        t = sess.submit(slots[j], _pinned(q), k)
        reqs.append((t, j, q, k))
    with pytest.raises(lcp.LcpError) as e:  # 1M queries x k=100 can never fit 8 MB
        sess.submit(slots[0], _pinned(np.zeros((100_000, 16), np.uint16)), 100)
    assert e.value.code == lcp.LCP_ERR_BUDGET
    for n, (t, j, q, k) in enumerate(reqs):
        ids, lc = sess.result(t)
        alone = lcp.lcp_topk_batch(idxs[j], _dev(q), k)
        assert np.array_equal(ids.numpy(), alone[0].cpu().numpy()), n
        assert np.array_equal(lc.numpy(), alone[1].cpu().numpy()), n
        if n % 10 == 0:
            w_ids, w_lcp = oracle.topk_batch(data[j][0], q[:50], k)
            assert np.array_equal(ids.numpy()[:50], w_ids) and np.array_equal(lc.numpy()[:50], w_lcp)
    st = sess.stats()
    assert st["completed"] == 60 and st["rejected"] == 1 and st["inflight"] == 0
    assert st["mem_peak"] <= 8 << 20
    assert sess.close() == lcp.LCP_OK
    for ix in idxs:
        assert lcp.lcp_index_sync(ix) == 0
        ix.close()


def test_session_request_filling_the_budget(lcp):
    """A request whose memory is the whole budget waits until every earlier
    request has retired, is then admitted, and the small requests behind it
    follow; every result equals the request served alone."""
    S = W.zipf_prefix_rows(20_000, 16, 1024, 1.1, 7)
    Qs = W.zipf_prefix_queries(S, 3_000, 1024, 1.1, 7)
    ix = lcp.lcp_index_build(_dev(S), max_k=10)
    k, Qbig = 10, 2_000
    budget = Qbig * (S.shape[1] * S.itemsize + 16 + 5 * k)  # the big request exactly
    sess = lcp.Session(mem_budget=budget, max_inflight=4, streams=2)
    slot = sess.add_index(ix)
    plan = [(0, 7), (7, 1), (100, 33), (200, Qbig), (7, 3), (900, 64), (50, 5)]
    tickets = [(sess.submit(slot, _pinned(Qs[o:o + q]), k), o, q) for o, q in plan]
    for t, o, q in tickets:
        ids, lc = sess.result(t)
        alone = lcp.lcp_topk_batch(ix, _dev(Qs[o:o + q]), k)
        assert np.array_equal(ids.numpy(), alone[0].cpu().numpy()), (o, q)
        assert np.array_equal(lc.numpy(), alone[1].cpu().numpy()), (o, q)
    st = sess.stats()
    assert st["completed"] == len(plan) and st["mem_peak"] <= budget and st["mem_in_use"] == 0
    assert sess.close() == lcp.LCP_OK
    ix.close()


def test_session_takes_device_and_host_buffers(lcp):
    """Queries and outputs may be device or host memory (the session copies
    with unified addressing); mixed requests give the same bytes as the
    request served alone."""
    S = W.zipf_prefix_rows(30_000, 32, 1024, 1.1, 8)
    Qs = W.zipf_prefix_queries(S, 2_000, 1024, 1.1, 8)
    ix = lcp.lcp_index_build(_dev(S), max_k=32)
    sess = lcp.Session(mem_budget=16 << 20, max_inflight=8, streams=4)
    slot = sess.add_index(ix)
    dq = _dev(Qs)
    plan = [(0, 500, True), (500, 1, False), (501, 700, True), (1201, 64, False), (1265, 735, True)]
    tickets = []
    for o, q, on_dev in plan:
        src = dq[o:o + q] if on_dev else _pinned(Qs[o:o + q])
        tickets.append((sess.submit(slot, src, 32), o, q, on_dev))
    for t, o, q, on_dev in tickets:
        ids, lc = sess.result(t)
        assert ids.is_cuda == on_dev and lc.is_cuda == on_dev
        alone = lcp.lcp_topk_batch(ix, dq[o:o + q], 32)
        assert torch.equal(ids.cpu(), alone[0].cpu()) and torch.equal(lc.cpu(), alone[1].cpu()), (o, q)
    w_ids, w_lcp = oracle.topk_batch(S, Qs[:40], 32)
    ids, lc = sess.result(sess.submit(slot, dq[:40], 32))
    assert np.array_equal(ids.cpu().numpy(), w_ids) and np.array_equal(lc.cpu().numpy(), w_lcp)
    assert sess.close() == lcp.LCP_OK
    ix.close()


def test_session_scan_slot_equals_scan_alone_and_index(lcp):
    """A full-scan slot (resident tokens, no index) served beside an index
    slot over the same rows: every request equals lcp_scan_topk alone, the
    index's answer and, on a sample, the oracle."""
    S = W.zipf_prefix_rows(60_000, 32, 1024, 1.1, 9)
    Qs = W.zipf_prefix_queries(S, 3_000, 1024, 1.1, 9)
    dS = _dev(S)
    ix = lcp.lcp_index_build(dS, max_k=64)
    sess = lcp.Session(mem_budget=32 << 20, max_inflight=6, streams=3)
    si = sess.add_index(ix)
    ss = sess.add_scan(dS)
    rng = np.random.default_rng(10)
    reqs = []
    for _ in range(24):
        Q = int(np.exp(rng.uniform(0, np.log(1500))))
        k = int(rng.choice([1, 10, 64]))
        o = int(rng.integers(0, 3_000 - Q))
        slot = int(rng.choice([si, ss]))
        reqs.append((sess.submit(slot, _pinned(Qs[o:o + Q]), k), slot, o, Q, k))
    for t, slot, o, Q, k in reqs:
        ids, lc = sess.result(t)
        a = lcp.lcp_scan_topk(dS, _dev(Qs[o:o + Q]), k)
        b = lcp.lcp_topk_batch(ix, _dev(Qs[o:o + Q]), k)
        assert np.array_equal(ids.numpy(), a[0].cpu().numpy()) and np.array_equal(lc.numpy(), a[1].cpu().numpy())
        assert np.array_equal(ids.numpy(), b[0].cpu().numpy()) and np.array_equal(lc.numpy(), b[1].cpu().numpy())
    w_ids, w_lcp = oracle.topk_batch(S, Qs[:30], 64)
    ids, lc = sess.result(sess.submit(ss, _pinned(Qs[:30]), 64))
    assert np.array_equal(ids.numpy(), w_ids) and np.array_equal(lc.numpy(), w_lcp)
    assert sess.close() == lcp.LCP_OK
    ix.close()
