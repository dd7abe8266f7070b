"""The five configured workloads against the CPU oracle, bit for bit.

Definition "Top-k LCP Retrieval" (Sec. 2.1) fixes one answer per query (the
key (-LCP, id) is unique) and Theorem 7 (Determinism) asks for the same bytes
on every run, alone or in a mix.  Each test below runs one workload at its
configured shape and size through the CUDA library and compares ids AND LCPs
with the oracle (`oracle.topk_batch`, the plain definition on the host):

* tree16_u8    -- every query, indexed and full scan (test_gpu_parity.py).
* zipf500k_L32 -- all 100,000 queries, indexed and full scan.
* zipf2m_L64   -- a seeded subset of 20,480 of the 1,000,000 queries against
                  the oracle; all 1,000,000 indexed answers against the GPU
                  full scan (itself checked on the subset).
* gnc1000      -- the 1,000-step insert-then-query stream, as direct calls
                  and as graph steps: every step t <= 50, every 50th step and
                  the last against the oracle, direct == graph on every step,
                  and the final 1,000,000-row index == the oracle's sorted
                  index == a fresh build.
* serving6     -- the six resident indexes; a seeded prefix of the Poisson
                  request stream through the serving session and through the
                  persistent work queue; every request equal to the same
                  request served alone, and a seeded sample of requests equal
                  to the oracle (ids and LCPs).
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


def pinned(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a).pin_memory()


def assert_same(got, want, what):
    gi, gl = got
    wi, wl = want
    assert gi.shape == wi.shape and gl.shape == wl.shape, "%s: shapes %s vs %s" % (what, gi.shape, wi.shape)
    if not (np.array_equal(gi, wi) and np.array_equal(gl, wl)):
        bad = np.nonzero((gi != wi).any(1) | (gl != wl).any(1))[0]
        r = bad[0]
        raise AssertionError("%s: %d/%d queries differ; first q=%d\n got ids %s lcp %s\nwant ids %s lcp %s"
                             % (what, len(bad), len(gi), r, gi[r][:16], gl[r][:16], wi[r][:16], wl[r][:16]))


def np_out(pair):
    return pair[0].cpu().numpy(), pair[1].cpu().numpy()


def test_zipf500k_L32_all_queries(lcp):
    """All 100,000 queries, indexed and full scan, against the oracle."""
    S, Qs, k = W.make_dataset("zipf500k_L32")
    assert S.shape == (500_000, 32) and Qs.shape == (100_000, 32) and k == 32
    idx = lcp.lcp_index_build(dev(S), max_k=k)
    dq = dev(Qs)
    got = np_out(lcp.lcp_topk_batch(idx, dq, k))
    sgot = np_out(lcp.lcp_scan_topk(dev(S), dq, k))
    torch.cuda.synchronize()
    assert lcp.lcp_index_sync(idx) == 0 and lcp.lcp_device_status() == 0
    idx.close()
    want = oracle.topk_batch(S, Qs, k)
    assert_same(got, want, "zipf500k_L32 indexed vs oracle (all 100,000 queries)")
    assert_same(sgot, want, "zipf500k_L32 full scan vs oracle (all 100,000 queries)")


C3_ORACLE_QUERIES = 20_480


def test_zipf2m_L64_oracle_subset_and_full_scan(lcp):
    """The bench workload: a seeded subset of 20,480 queries against the
    oracle (indexed and full scan), all 1,000,000 indexed answers against the
    full scan of the same batch."""
    S, Qs, k = W.make_dataset("zipf2m_L64")
    assert S.shape == (2_000_000, 64) and Qs.shape == (1_000_000, 64) and k == 100
    idx = lcp.lcp_index_build(dev(S), max_k=k)
    dq = dev(Qs)
    got = np_out(lcp.lcp_topk_batch(idx, dq, k))
    sgot = np_out(lcp.lcp_scan_topk(dev(S), dq, k))
    torch.cuda.synchronize()
    assert lcp.lcp_index_sync(idx) == 0 and lcp.lcp_device_status() == 0
    idx.close()
    assert_same(got, sgot, "zipf2m_L64 indexed vs full scan (all 1,000,000 queries)")
    pick = np.sort(np.random.default_rng(2024).choice(len(Qs), C3_ORACLE_QUERIES, replace=False))
    want = oracle.topk_batch(S, Qs[pick], k)
    assert_same((got[0][pick], got[1][pick]), want, "zipf2m_L64 indexed vs oracle (20,480 queries)")
    assert_same((sgot[0][pick], sgot[1][pick]), want, "zipf2m_L64 full scan vs oracle (20,480 queries)")


def _gnc_checked(t):
    """Steps (1-based) compared with the oracle: t <= 50, every 50th, the last."""
    return t <= 50 or t % 50 == 0 or t == 1000


def test_gnc1000_stream_direct_and_graph(lcp):
    w = W.WORKLOADS["gnc1000"]
    steps_n, k = w["steps"], w["k"]
    g = W.GncStream(sensors=w["sensors"], seed=w["seed"])
    steps = [g.step() for _ in range(steps_n)]
    dsteps = dev(np.stack(steps))
    outs = {}
    finals = {}
    for mode in ("direct", "graph"):
        ix = lcp.lcp_index_build(torch.zeros((0, 8), dtype=torch.int16, device="cuda"), max_k=k,
                                 capacity=steps_n * w["sensors"])
        st = lcp.Step(ix, w["sensors"], w["sensors"], k) if mode == "graph" else None
        all_ids = torch.empty((steps_n, w["sensors"], k), dtype=torch.int32, device="cuda")
        all_lcp = torch.empty((steps_n, w["sensors"], k), dtype=torch.uint8, device="cuda")
        for t in range(steps_n):
            if st is None:
                lcp.lcp_index_insert(ix, dsteps[t])
                lcp.lcp_topk_batch(ix, dsteps[t], k, all_ids[t], all_lcp[t])
            else:
                st.run(dsteps[t], dsteps[t], all_ids[t], all_lcp[t])
        torch.cuda.synchronize()
        assert lcp.lcp_index_sync(ix) == 0
        assert ix.N == steps_n * w["sensors"]
        outs[mode] = (all_ids.cpu().numpy(), all_lcp.cpu().numpy())
        finals[mode] = np_out(lcp.lcp_index_export(ix))
        if st is not None:
            st.close()
        ix.close()
    assert np.array_equal(outs["direct"][0], outs["graph"][0]) and np.array_equal(outs["direct"][1],
                                                                                  outs["graph"][1])
    S_all = np.concatenate(steps)
    checked = [t for t in range(1, steps_n + 1) if _gnc_checked(t)]
    assert len(checked) == 69
    for t in checked:
        want = oracle.topk_batch(S_all[: t * w["sensors"]], steps[t - 1], k)
        for mode in ("direct", "graph"):
            assert_same((outs[mode][0][t - 1], outs[mode][1][t - 1]), want, "gnc step %d (%s)" % (t, mode))
    # insert == rebuild at N = 1,000,000: the oracle's sorted index and a fresh build
    w_ids, w_H = oracle.sorted_index(S_all)
    fresh = lcp.lcp_index_build(dev(S_all), max_k=k)
    f_ids, f_H = np_out(lcp.lcp_index_export(fresh))
    torch.cuda.synchronize()
    assert lcp.lcp_index_sync(fresh) == 0
    fresh.close()
    assert np.array_equal(f_ids, w_ids) and np.array_equal(f_H, w_H)
    for mode in ("direct", "graph"):
        assert np.array_equal(finals[mode][0], w_ids), mode
        assert np.array_equal(finals[mode][1], w_H), mode


SERVING_REQUESTS = 2_000
SERVING_ORACLE_SAMPLE = 48
ORACLE_PAIRS_PER_REQUEST = 150_000_000  # query-row LCPs per sampled request, at most


def _serving_setup(lcp):
    w = W.WORKLOADS["serving6"]
    data, indexes = [], []
    for i, (N, L) in enumerate(W.SERVING_INDEXES):
        S = W.zipf_prefix_rows(N, L, w["vocab"], w["s"], w["seed"] * 100 + i)
        pool = W.zipf_prefix_queries(S, 16_384, w["vocab"], w["s"], w["seed"] * 100 + i)
        data.append((S, pool))
        indexes.append(lcp.lcp_index_build(dev(S), max_k=100))
    rq = W.serving_requests(SERVING_REQUESTS, w["rate"], len(indexes), w["seed"])
    rng = np.random.default_rng(w["seed"])
    reqs = []
    for i in range(SERVING_REQUESTS):
        j, Q, k = int(rq["index"][i]), int(rq["n_queries"][i]), int(rq["k"][i])
        qoff = int(rng.integers(0, 16_384 - Q + 1))
        reqs.append((float(rq["arrival_s"][i]), j, qoff, Q, k))
    return data, indexes, reqs


def _oracle_sample(data, reqs, getters):
    """A seeded sample of requests against the oracle: every query of the
    request when Q x N stays under ORACLE_PAIRS_PER_REQUEST, else a seeded
    subset of its queries.  `getters` maps a path name to a function giving
    request i's (ids, lcp) as numpy arrays."""
    rng = np.random.default_rng(77)
    sample = np.sort(rng.choice(len(reqs), SERVING_ORACLE_SAMPLE, replace=False))
    for i in sample:
        _, j, qoff, Q, k = reqs[i]
        S, pool = data[j]
        q = pool[qoff:qoff + Q]
        rows = np.arange(Q)
        cap = max(1, ORACLE_PAIRS_PER_REQUEST // len(S))
        if Q > cap:
            rows = np.sort(rng.choice(Q, cap, replace=False))
        want = oracle.topk_batch(S, q[rows], k)
        for what, get in getters.items():
            gi, gl = get(i)
            assert_same((gi[rows], gl[rows]), want,
                        "%s request %d (index %d, Q=%d, k=%d) vs oracle" % (what, i, j, Q, k))


def test_serving6_session_and_queue_equal_alone_and_oracle(lcp):
    data, indexes, reqs = _serving_setup(lcp)
    # the same request served alone, once per request (device buffers)
    dpools = [dev(p) for _, p in data]
    alone = []
    for (_, j, qoff, Q, k) in reqs:
        alone.append(lcp.lcp_topk_batch(indexes[j], dpools[j][qoff:qoff + Q], k))
    torch.cuda.synchronize()
    alone = [np_out(a) for a in alone]
    # output slots, 256-byte aligned: ids then LCPs
    offs, total = [], 0
    for (_, _, _, Q, k) in reqs:
        offs.append(total)
        total += (Q * k * 5 + 255) & ~255

    def slot(buf, i):
        _, _, _, Q, k = reqs[i]
        o = offs[i]
        ids = buf[o:o + Q * k * 4].view(torch.int32).view(Q, k)
        lc = buf[o + Q * k * 4:o + Q * k * 5].view(Q, k)
        return ids, lc

    # serving session: host queries and outputs, Poisson arrivals, memory budget
    ppools = [pinned(p) for _, p in data]
    arena = torch.zeros(total, dtype=torch.uint8).pin_memory()
    sess = lcp.Session(mem_budget=256 << 20, max_inflight=64, streams=8)
    slots = [sess.add_index(ix) for ix in indexes]
    rr = []
    for i, (arr, j, qoff, Q, k) in enumerate(reqs):
        ids, lc = slot(arena, i)
        qp = ppools[j].data_ptr() + qoff * ppools[j].shape[1] * 2
        rr.append(lcp.ReplayRequest(arr, slots[j], k, Q, qp, ids.data_ptr(), lc.data_ptr()))
    rc, lat, _ = sess.replay(rr, timeout_s=120.0)
    assert rc == 0 and (lat >= 0).all()
    assert sess.close() == 0
    for i in range(len(reqs)):
        got = tuple(x.numpy() for x in slot(arena, i))
        assert_same(got, alone[i], "session request %d vs alone" % i)
    # persistent work queue: device queries and outputs, same stream of requests
    darena = torch.zeros(total, dtype=torch.uint8, device="cuda")
    qr = []
    for i, (arr, j, qoff, Q, k) in enumerate(reqs):
        ids, lc = slot(darena, i)
        qp = dpools[j].data_ptr() + qoff * dpools[j].shape[1] * 2
        qr.append(lcp.QueueReplayRequest(arr, indexes[j].handle.value, k, Q, qp, ids.data_ptr(), lc.data_ptr()))
    torch.cuda.synchronize()
    qu = lcp.Queue(max_requests=1024, max_tasks=1 << 18, idle_ms=20.0)
    qrc, qlat, _ = qu.replay(qr, timeout_s=120.0)
    qu.close()
    assert qrc == 0 and (qlat >= 0).all()
    harena = darena.cpu()
    for i in range(len(reqs)):
        got = tuple(x.numpy() for x in slot(harena, i))
        assert_same(got, alone[i], "queue request %d vs alone" % i)
    _oracle_sample(data, reqs, {"session": lambda i: tuple(x.numpy() for x in slot(arena, i)),
                                "queue": lambda i: tuple(x.numpy() for x in slot(harena, i))})
    for ix in indexes:
        assert lcp.lcp_index_sync(ix) == 0
        ix.close()
