"""The allocation-free full scan (lcp_scan_topk_noalloc) gives exactly the
results of lcp_scan_topk, called through the C ABI.

That entry point exists for callers that cannot allocate device memory when
they call in (real-time loops that must not block in the allocator, code
limited to start-up allocation, host code inside a global-mode stream
capture); it runs on a fixed scratch array in the library's device image.
Two calls in a row on different inputs check that the second call is not
disturbed by what the first left in the shared scratch.  This file is
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


def test_noalloc_scan_matches_scan_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_04936_b300 as P
    lib = P.raw_lib()
    cases = [("zipf500k_L32", 200_000, 3_000, 32), ("tree16_u8", 10_000, 1_000, 10)]
    for name, N, Q, k in cases:
        S, Qs, _ = W.make_dataset(name, N=N, Q=Q)
        w = W.WORKLOADS[name]
        dS, dQ = _dev(S), _dev(Qs)
        want = _call(lib.lcp_scan_topk, P, dS, dQ, k, w["L"], w["token_bytes"], w["vocab"])
        got = _call(lib.lcp_scan_topk_noalloc, P, dS, dQ, k, w["L"], w["token_bytes"], w["vocab"])
        assert torch.equal(got[0], want[0]), name
        assert torch.equal(got[1], want[1]), name
    assert lib.lcp_device_status() == 0


def test_noalloc_rejects_requests_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_04936_b300 as P
    lib = P.raw_lib()
    cap = 32 << 20
    N = cap // 8  # plane 0 alone fills the scratch
    one = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    rc = lib.lcp_scan_topk_noalloc(one, N, P._Format(1, 8, 0), one, 1, 1, one, one, None)
    assert rc == P.LCP_ERR_INVALID
