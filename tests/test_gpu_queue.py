"""Persistent search fed by a work queue: requests of uneven size and k
against several resident indexes, all answered by one long-lived launch,
each equal to the same request served alone (and the oracle on a sample)."""
import time

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


def test_queue_mix_equals_alone(lcp):
    rng = np.random.default_rng(9)
    specs = [(3_000, 16, 1024, 1.1), (50_000, 32, 32768, 1.05), (200_000, 64, 32768, 1.05)]
    data, idxs = [], []
    for i, (N, L, V, s) in enumerate(specs):
        S = W.zipf_prefix_rows(N, L, V, s, 60 + i)
        Qs = W.zipf_prefix_queries(S, 6_000, V, s, 60 + i)
        data.append((S, dev(Qs), Qs))
        idxs.append(lcp.lcp_index_build(dev(S), max_k=100))
    torch.cuda.synchronize()
    qu = lcp.Queue(max_requests=16, max_tasks=4096, idle_ms=5.0)
    reqs, pending = [], []
    for r in range(80):
        j = int(rng.integers(0, 3))
        Q = int(np.exp(rng.uniform(0, np.log(3000))))
        k = int(rng.choice([1, 10, 100]))
        off = int(rng.integers(0, 6_000 - Q))
        while True:
            try:
                t = qu.submit(idxs[j], data[j][1][off:off + Q], k)
                break
            except lcp.LcpError as e:
                assert e.code == lcp.LCP_ERR_CAPACITY
                assert qu.poll(pending.pop(0), 10_000) == lcp.LCP_OK
        pending.append(t)
        reqs.append((t, j, off, Q, k))
    for n, (t, j, off, Q, k) in enumerate(reqs):
        ids, lc = qu.result(t)
        alone = lcp.lcp_topk_batch(idxs[j], data[j][1][off:off + Q], k)
        assert torch.equal(ids, alone[0]) and torch.equal(lc, alone[1]), n
        if n % 10 == 0:
            w_ids, w_lcp = oracle.topk_batch(data[j][0], data[j][2][off:off + min(Q, 40)], k)
            assert np.array_equal(ids[:40].cpu().numpy(), w_ids) and np.array_equal(lc[:40].cpu().numpy(), w_lcp)
    st = qu.stats()
    assert st["inflight"] == 0 and st["worker_launches"] >= 1
    qu.close()
    assert lcp.lcp_device_status() == 0
    for ix in idxs:
        ix.close()


def test_queue_worker_idles_out_and_relaunches(lcp):
    S, Qs, k = W.make_dataset("tree16_u8", N=5_000, Q=400)
    idx = lcp.lcp_index_build(dev(S), max_k=k)
    dq = dev(Qs)
    torch.cuda.synchronize()
    qu = lcp.Queue(idle_ms=1.0)
    want = lcp.lcp_topk_batch(idx, dq, k)
    for rep in range(3):
        ids, lc = qu.result(qu.submit(idx, dq, k))
        assert torch.equal(ids, want[0]) and torch.equal(lc, want[1])
        time.sleep(0.05)  # far past idle_ms: every warp has left
    assert qu.stats()["worker_launches"] >= 2
    # an empty request completes at once
    t = qu.submit(idx, dq[:0], k)
    assert qu.poll(t) == lcp.LCP_OK
    with pytest.raises(lcp.LcpError):
        qu.submit(idx, dq, k + 100)  # k above the index's max_k
    qu.close()
    idx.close()


def test_queue_replay_open_loop(lcp):
    """The native open-loop driver: Poisson arrivals, every request completes
    with a non-negative latency and its outputs equal the request alone."""
    rng = np.random.default_rng(3)
    S, Qs, k = W.make_dataset("zipf500k_L32", N=30_000, Q=4_000)
    idx = lcp.lcp_index_build(dev(S), max_k=k)
    dq = dev(Qs)
    n = 200
    arr = np.cumsum(rng.exponential(1 / 20_000, n))
    sizes = np.exp(rng.uniform(0, np.log(1000), n)).astype(int)
    offs = [int(rng.integers(0, 4_000 - q)) for q in sizes]
    outs = [(torch.empty((q, k), dtype=torch.int32, device="cuda"),
             torch.empty((q, k), dtype=torch.uint8, device="cuda")) for q in sizes]
    reqs = [lcp.QueueReplayRequest(float(arr[i]), idx.handle.value, k, int(sizes[i]),
                                   dq[offs[i]:].data_ptr(), outs[i][0].data_ptr(), outs[i][1].data_ptr())
            for i in range(n)]
    torch.cuda.synchronize()
    qu = lcp.Queue(max_requests=32, max_tasks=2048, idle_ms=2.0)
    rc, lat, wall = qu.replay(reqs, timeout_s=30.0)
    assert rc == lcp.LCP_OK and (lat >= 0).all() and wall > 0
    qu.close()
    for i in range(n):
        alone = lcp.lcp_topk_batch(idx, dq[offs[i]:offs[i] + sizes[i]], k)
        assert torch.equal(outs[i][0], alone[0]) and torch.equal(outs[i][1], alone[1]), i
    idx.close()
