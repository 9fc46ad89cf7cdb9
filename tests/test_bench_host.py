"""Host-side pieces of bench.py, checked on the CPU: the combined integer roofline it reports
against (derived from the unit counts, not measured here), and its reading of the committed
ncu summary (the traffic and counters it attaches only for the profiled launch shape)."""
import sys

import pytest

import bench


def test_roofline_peak_from_unit_counts():
    # the LDS pipe bounds the T-table path at 32 / 160 blocks per SM-clock; that uses
    # 160 x 240 / 160 = 48 of the 64 ALU lanes, and the other 16 lanes run gates at 356.25
    # lane-operations per block
    t = 32.0 / 160.0
    b = (64.0 - 240.0 * t) / (22800.0 / 64.0)
    assert bench.blocks_per_sm_clock() == pytest.approx(t + b, rel=1e-12)
    assert bench.roofline_peak_gbs(152, 2070.0) == pytest.approx((t + b) * 152 * 2.07e9 * 16 / 1e9, rel=1e-12)
    assert 1232 < bench.roofline_peak_gbs(152, 2070.0) < 1234


def test_profile_summary_is_readable():
    prof = bench.read_profile()
    assert prof["shape"] is not None and all(v > 0 for v in prof["shape"])
    for d in ("encrypt", "decrypt"):
        # DRAM bytes per 2^26-block launch: at least input plus most of the output (1 GiB each)
        assert 1.5e9 < prof["traffic"][d] < 2.5e9
        c = prof["ncu"][d]
        assert {"lsu_pipe_pct", "alu_pipe_pct", "shared_bank_conflict_pct", "warps_active_pct", "dram_gbs"} <= set(c)
        assert 0 < c["lsu_pipe_pct"] <= 100 and 0 < c["alu_pipe_pct"] <= 100


def test_default_arguments_are_one_gpu(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse_args()
    assert a.gpus == 1 and a.impl == "ours" and a.warmup >= 3 and a.steps >= 1
