"""Serving-session admission policy without a GPU (dry-run sessions).

In a dry run a request needs Q * (16 + 5k) bytes, is admitted in arrival
order while fewer than max_inflight are in flight and its bytes fit the
budget, and completes on the next poll.  These tests fault nothing: the
failure paths are host-side (budget rejection, cancellation at shutdown,
invalid tickets)."""
import numpy as np
import pytest

import paper_2602_04936_b300 as P


def _req(Q, k):
    return (np.zeros((Q, 4), np.uint8), np.zeros((Q, k), np.int32), np.zeros((Q, k), np.uint8))


def _submit(s, slot, Q, k):
    import torch
    q, i, l = _req(Q, k)
    return s.submit(slot, torch.from_numpy(q), k, torch.from_numpy(i), torch.from_numpy(l))


def test_invalid_configs_rejected():
    for cfg in [(0, 4, 1), (1000, 0, 1), (1000, 4, 0), (1000, 4, 65)]:
        with pytest.raises(P.LcpError) as e:
            P.Session(*cfg, dry_run=True)
        assert e.value.code == P.LCP_ERR_INVALID


def test_budget_admission_fifo_and_rejection():
    s = P.Session(mem_budget=10_000, max_inflight=8, streams=2, dry_run=True)
    slot = s.add_index(None)
    a = _submit(s, slot, 50, 10)    # 3,300 bytes: admitted
    b = _submit(s, slot, 100, 10)   # 6,600: admitted (9,900 in use)
    c = _submit(s, slot, 10, 10)    # 660: waits, the budget is full
    with pytest.raises(P.LcpError) as e:
        _submit(s, slot, 200, 10)   # 13,200 > budget: can never fit
    assert e.value.code == P.LCP_ERR_BUDGET
    st = s.stats()
    assert (st["submitted"], st["admitted"], st["rejected"]) == (4, 2, 1)
    assert (st["inflight"], st["pending"], st["mem_in_use"]) == (2, 1, 9_900)
    assert st["mem_peak"] == 9_900
    # polling retires a and b, which admits c
    assert s.poll(a) == P.LCP_OK
    st = s.stats()
    assert st["admitted"] == 3 and st["pending"] == 0
    assert s.poll(b) == P.LCP_OK and s.poll(c) == P.LCP_OK
    assert s.poll(a) == P.LCP_ERR_INVALID  # a ticket reports once
    assert s.stats()["completed"] == 3 and s.stats()["mem_in_use"] == 0
    assert s.close() == P.LCP_OK


def test_inflight_limit_and_arrival_order():
    s = P.Session(mem_budget=1 << 30, max_inflight=1, streams=1, dry_run=True)
    slot = s.add_index(None)
    t = [_submit(s, slot, 4, 1) for _ in range(5)]
    st = s.stats()
    assert st["inflight"] == 1 and st["pending"] == 4
    # a large request behind small ones waits its turn (no overtaking)
    big = _submit(s, slot, 1000, 100)
    for i, ticket in enumerate(t):
        assert s.poll(ticket) == P.LCP_OK
        assert s.stats()["admitted"] == i + 2
    assert s.poll(big) == P.LCP_OK
    assert s.close() == P.LCP_OK


def test_shutdown_cancels_waiting_requests():
    s = P.Session(mem_budget=1000, max_inflight=1, streams=1, dry_run=True)
    slot = s.add_index(None)
    for _ in range(3):
        _submit(s, slot, 2, 1)
    st = s.stats()
    assert st["inflight"] == 1 and st["pending"] == 2
    assert s.close() == P.LCP_OK


def test_bad_submissions():
    s = P.Session(mem_budget=1000, max_inflight=1, streams=1, dry_run=True)
    slot = s.add_index(None)
    with pytest.raises(P.LcpError):
        _submit(s, slot + 1, 2, 1)      # unknown slot
    with pytest.raises(P.LcpError):
        _submit(s, slot, 2, 0)          # k < 1
    assert s.poll(12345) == P.LCP_ERR_INVALID
    s.close()


def test_replay_driver_dry_run():
    """The open-loop driver submits each request at its time and records a
    non-negative latency; an over-budget request is marked -1."""
    s = P.Session(mem_budget=10_000, max_inflight=4, streams=2, dry_run=True)
    slot = s.add_index(None)
    q = np.zeros((64, 4), np.uint8)
    ids = np.zeros((64, 10), np.int32)
    lc = np.zeros((64, 10), np.uint8)
    reqs = []
    for i in range(20):
        Q = 200 if i == 7 else 8      # request 7 needs 13,200 bytes > budget
        reqs.append(P.ReplayRequest(i * 0.001, slot, 10, Q, q.ctypes.data, ids.ctypes.data,
                                    lc.ctypes.data))
    rc, lat, wall = s.replay(reqs, timeout_s=10.0)
    assert rc == P.LCP_OK
    assert lat[7] == -1.0
    assert (np.delete(lat, 7) >= 0).all()
    assert wall >= 0.018
    assert s.stats()["rejected"] == 1 and s.stats()["completed"] == 19
    s.close()
