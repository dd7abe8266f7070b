"""C-ABI checks that need no GPU: the library builds and loads, exports every
entry point include/lcp.h declares, and rejects bad arguments synchronously
(LCP_ERR_INVALID) before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lcp.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"LCP_API\s+[\w\s\*]+?\b(lcp_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lcp():
    import paper_2602_04936_b300 as P
    return P


def test_header_declares_the_abi(lcp):
    names = _declared()
    for must in ("lcp_index_build", "lcp_index_insert", "lcp_topk_batch", "lcp_scan_topk",
                 "lcp_index_destroy", "lcp_status_string"):
        assert must in names
    assert sorted(lcp.ABI_SYMBOLS) == names


def test_library_exports_every_declared_symbol(lcp):
    out = subprocess.run(["nm", "-D", "--defined-only", lcp.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lcp_\w+)", out))
    for name in _declared():
        assert name in exported, name
        assert getattr(lcp.raw_lib(), name) is not None


def test_status_strings(lcp):
    assert lcp.lcp_status_string(0) == "ok"
    assert "invalid" in lcp.lcp_status_string(lcp.LCP_ERR_INVALID)
    assert "capacity" in lcp.lcp_status_string(lcp.LCP_ERR_CAPACITY)
    assert "timed out" in lcp.lcp_status_string(lcp.LCP_ERR_TIMEOUT)


def test_invalid_arguments_rejected_without_device(lcp):
    L = lcp.raw_lib()
    F = lcp._Format
    h = ctypes.c_void_p()
    one = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    # bad token width, bad L, k out of range, null output handle
    assert L.lcp_index_build(one, 10, F(3, 8, 0), 0, 10, None, ctypes.byref(h)) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_build(one, 10, F(2, 0, 0), 0, 10, None, ctypes.byref(h)) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_build(one, 10, F(2, 256, 0), 0, 10, None, ctypes.byref(h)) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_build(one, 10, F(2, 8, 0), 0, 0, None, ctypes.byref(h)) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_build(one, 10, F(2, 8, 0), 0, 129, None, ctypes.byref(h)) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_build(one, 10, F(2, 8, 0), 5, 10, None, ctypes.byref(h)) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_build(None, 10, F(2, 8, 0), 0, 10, None, ctypes.byref(h)) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_build(one, 10, F(2, 8, 0), 0, 10, None, None) == lcp.LCP_ERR_INVALID
    assert L.lcp_scan_topk(one, 10, F(1, 8, 0), one, 4, 0, one, one, None) == lcp.LCP_ERR_INVALID
    assert L.lcp_scan_topk(one, 10, F(1, 8, 0), one, 4, 1025, one, one, None) == lcp.LCP_ERR_INVALID
    assert L.lcp_scan_topk(one, 10, F(1, 8, 0), None, 4, 3, one, one, None) == lcp.LCP_ERR_INVALID
    assert L.lcp_topk_batch(None, one, 4, 3, one, one, None) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_insert(None, one, 4, None) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_size(None, None, None) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_sync(None) == lcp.LCP_ERR_INVALID
    assert L.lcp_index_destroy(None) == lcp.LCP_OK
    assert L.lcp_debug_bounded_wait(0, None) == lcp.LCP_ERR_INVALID


def test_launch_counter_starts_at_zero_without_work(lcp):
    assert lcp.lcp_launch_count() >= 0
