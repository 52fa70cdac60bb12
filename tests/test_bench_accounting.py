"""bench.py's roofline accounting on the CPU: the numerator counts only the algorithm's
own arithmetic (Sec. IV-C Step 2, Tables I-II), and ncu counters are reported only for
the kernel sources they were taken on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2305_05286_gb300 import inputs as I  # noqa: E402


def test_cbp_sp_counts_two_phi_and_the_simple_operations():
    # per edge: 2 phi (20 each) + 8 simple operations + 1 syndrome XOR; per variable:
    # phi + 4 (the flushed posterior of Eq. s4e20 and the decision of Eq. s2e7)
    assert bench.OPS_EDGE["cbp_sp"] + bench.OPS_SYN == 49
    assert bench.OPS_VAR["cbp_sp"] == 24


def test_fraction_of_a_known_run():
    # a run of 65536 frames of the 26112-bit code with 261396 frame-sweeps in 180.33 ms
    # at 2070 MHz on 152 SMs: (3.694e10 edge-sweeps * 49 + 6.83e9 variable-sweeps * 24)
    # / 0.18033 s / 40.27 T lane-ops/s = 0.27
    qc = I.code_26112()
    st = {"sweeps_total": 261396}
    peak = 152 * 128 * 2070e6 / 1e12
    r = bench.roofline_entry("cbp_sp", qc, st, 180.33, peak, "26112", None)
    assert r["units"]["edge_sweeps"] == 36938391552
    assert abs(r["frac"] - 0.2717) < 1e-3
    assert r["bound"] == "alu" and r["unit"] == "T lane-ops/s"


def test_counters_only_for_the_sources_they_were_taken_on(monkeypatch):
    qc = I.code_26112()
    st = {"sweeps_total": 1000}
    cap = {"kernel": "k", "date": "d", "frames": 2432, "sources": bench.kernel_source_hash("cbp_sp"),
           "dram_bytes_per_frame_sweep": 1.5e6, "thread_inst_per_edge_sweep": 80.0,
           "issue_active": 0.6, "warps_active_per_sm": 24.0}
    monkeypatch.setitem(bench.CAPTURES, "cbp_sp", cap)
    r = bench.roofline_entry("cbp_sp", qc, st, 1.0, 40.0, "26112", None)
    assert r["traffic"] == 1.5e9 and r["kernel_counters"]["thread_inst_per_edge_sweep"] == 80.0
    # another code, or changed sources: no traffic and no counters
    assert bench.roofline_entry("cbp_sp", qc, st, 1.0, 40.0, "576", None)["traffic"] is None
    monkeypatch.setitem(bench.CAPTURES, "cbp_sp", dict(cap, sources="0" * 16))
    r = bench.roofline_entry("cbp_sp", qc, st, 1.0, 40.0, "26112", None)
    assert r["traffic"] is None and r["kernel_counters"] is None
