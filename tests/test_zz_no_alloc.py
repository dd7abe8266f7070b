"""The allocation-free full scan (lcp_scan_topk_noalloc) gives exactly the
results of lcp_scan_topk, called through the C ABI.

That entry point exists for callers that cannot allocate device memory when
they call in (real-time loops that must not block in the allocator, code
limited to start-up allocation, host code inside a global-mode stream
capture); it runs on a fixed scratch array in the library's device image.
Calls in a row on different inputs check that each call is not disturbed by
what the one before left in the shared scratch; a sample of each call's
queries is also checked against the CPU oracle.  This file is
collected last so that a failure here cannot hide another test's result.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(a).cuda()


def _call(fn, P, S, Qs, k, L_tokens, tb, vocab):
    Q = Qs.shape[0]
    ids = torch.full((Q, k), 7, dtype=torch.int32, device="cuda")   # not -1/0: must be overwritten
    lc = torch.full((Q, k), 9, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.c_void_p(S.data_ptr()), S.shape[0], P._Format(tb, L_tokens, vocab),
            ctypes.c_void_p(Qs.data_ptr()), Q, k, ctypes.c_void_p(ids.data_ptr()),
            ctypes.c_void_p(lc.data_ptr()), stream)
    assert rc == 0, P.lcp_status_string(rc)
    torch.cuda.synchronize()
    return ids, lc


SCRATCH = 32 << 20


def _need(N, Q, k):
    """Scratch bytes of one call: the rows' first words in two halves, then
    one N-slice of per-query counts and logs of k + 64 keys."""
    return 2 * ((N * 4 + 255) & ~255) + ((Q * 4 + 255) & ~255) + Q * (k + 64) * 8


def _max_queries(N, k):
    """Largest batch that fits the scratch."""
    Q = (SCRATCH - 2 * ((N * 4 + 255) & ~255)) // ((k + 64) * 8 + 4)
    while _need(N, Q + 1, k) <= SCRATCH:
        Q += 1
    while _need(N, Q, k) > SCRATCH:
        Q -= 1
    return Q


# (workload, N, Q, k): the per-thread-log path on both sides; one and 32
# queries (where lcp_scan_topk takes the threshold selection instead, the more
# independent comparison); k = 1,024 (a merge CTA takes 4 lists, so at most 4
# slices); a batch of 3,000 queries over 2M rows, where the scratch caps the
# slice count below what the rows would allow; and the largest batch that
# fits next to a 2M-row plane (one slice, just under the limit).
CASES = [("zipf500k_L32", 200_000, 3_000, 32), ("tree16_u8", 10_000, 1_000, 10),
         ("zipf500k_L32", 200_000, 1, 32), ("tree16_u8", 10_000, 32, 10),
         ("tree16_u8", 10_000, 300, 1024), ("zipf500k_L32", 2_000_000, 3_000, 100),
         ("zipf500k_L32", 2_000_000, _max_queries(2_000_000, 100), 100)]


def test_noalloc_scan_matches_scan_and_oracle_call_after_call():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2602_04936_b300 as P
    lib = P.raw_lib()
    rng = np.random.default_rng(31)
    for name, N, Q, k in CASES:
        S, Qs, _ = W.make_dataset(name, N=N, Q=Q)
        w = W.WORKLOADS[name]
        dS, dQ = _dev(S), _dev(Qs)
        want = _call(lib.lcp_scan_topk, P, dS, dQ, k, w["L"], w["token_bytes"], w["vocab"])
        got = _call(lib.lcp_scan_topk_noalloc, P, dS, dQ, k, w["L"], w["token_bytes"], w["vocab"])
        assert torch.equal(got[0], want[0]), (name, N, Q, k)
        assert torch.equal(got[1], want[1]), (name, N, Q, k)
        pick = np.sort(rng.choice(Q, min(Q, 12), replace=False))
        w_ids, w_lcp = oracle.topk_batch(S, Qs[pick], k)
        assert np.array_equal(got[0].cpu().numpy()[pick], w_ids), (name, N, Q, k)
        assert np.array_equal(got[1].cpu().numpy()[pick], w_lcp), (name, N, Q, k)
    assert lib.lcp_device_status() == 0


def test_noalloc_rejects_requests_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_04936_b300 as P
    lib = P.raw_lib()
    N = SCRATCH // 8  # plane 0 alone fills the scratch
    one = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    rc = lib.lcp_scan_topk_noalloc(one, N, P._Format(1, 8, 0), one, 1, 1, one, one, None)
    assert rc == P.LCP_ERR_INVALID
    # one query more than the largest batch that fits beside a 2M-row plane
    Q = _max_queries(2_000_000, 100) + 1
    rc = lib.lcp_scan_topk_noalloc(one, 2_000_000, P._Format(2, 32, 0), one, Q, 100, one, one, None)
    assert rc == P.LCP_ERR_INVALID
