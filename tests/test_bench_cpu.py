"""The bench's roofline arithmetic, on the host: the byte and instruction
models behind the reported fractions (no GPU, no measurement)."""
import math

import numpy as np
import pytest

import bench


@pytest.mark.parametrize("k,a_mean", [(1, 0.0), (100, 15.9), (100, 0.0), (1024, 700.5)])
def test_answer_and_fill_count_every_output_byte_once(k, a_mean):
    """The answer kernel writes the |A| first results, the fill the other
    k - |A|: 5 bytes a result (4-byte id + 1-byte LCP) between them."""
    ans = bench.answer_algorithmic_bytes(k, a_mean)
    fill = bench.fill_algorithmic_bytes(k, a_mean)
    inputs_and_records = 16 + (k + 2) + a_mean * 4 + 32 + 32 + (k - a_mean) * 4
    assert math.isclose(ans + fill - inputs_and_records, 5 * k)


def test_issue_roofline_formula(monkeypatch):
    """achieved = warp instructions a query x Q / launch time; peak = SMs x 4
    schedulers x 1 warp instruction a clock at the sampled clock."""
    monkeypatch.setattr(bench, "committed_inst_per_query", lambda kernel: 600.0)
    r = bench.issue_roofline("k_topk_answer", 1_000_000, 0.6, 2032.0, 148)
    ach = 600.0 * 1e6 / 0.6e-3
    pk = 148 * 4 * 2032e6
    assert math.isclose(r["frac"], round(ach / pk, 4))
    assert math.isclose(r["peak"], round(pk / 1e12, 4))
    monkeypatch.setattr(bench, "committed_inst_per_query", lambda kernel: None)
    assert bench.issue_roofline("k_topk_answer", 1_000_000, 0.6, 2032.0, 148) is None


def test_scan_models():
    """Integer-ALU model: 2 operations a (query, row) pair against 128 lanes
    a multiprocessor; byte model: rows once, queries and results."""
    r = bench.scan_alu_model(1024, 2_000_000, 0.45, 2032.0, 148)
    assert math.isclose(r["frac"], round(2 * 1024 * 2e6 / 0.45e-3 / (148 * 128 * 2032e6), 4))
    assert bench.scan_alu_model(1024, 2_000_000, 0.45, None, 148) is None
    h = bench.scan_hbm_model(1, 2_000_000, 16, 100, 0.1, 6500.0)
    assert h["bytes"] == 2_000_000 * 16 * 8 + 16 * 8 + 100 * 5
    assert h["fetch_bytes"] == 2_000_000 * 64 + 16 * 8 + 100 * 5


def test_build_kernel_bytes():
    """Row gather: id and row in, sorted row, its word 0 and H out."""
    m = bench.build_kernel_bytes(2_000_000, 64, 2, 16)
    assert m["k_gather_rows_lcp"] == 2_000_000 * (4 + 128 + 128 + 8 + 1)
    assert m["k_onesweep"] == 2_000_000 * 16 and m["k_tile_counts"] == 2_000_000 * 4
    assert m["k_keys_word0"] == 2_000_000 * 24


def test_locate_bytes_follow_bucket_sizes():
    """One 32-byte sector a binary-search level inside the query's
    first-token bucket (ceil(log2(size + 1)) levels)."""
    S = np.zeros((1023, 4), np.uint16)  # one bucket of 1,023 rows: 10 levels
    Qs = np.zeros((5, 4), np.uint16)
    assert bench.locate_algorithmic_bytes(S, Qs) == 4 * 2 + 32 + 10 * 32 + 16
