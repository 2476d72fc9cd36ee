"""CPU tests of bench.py's host-side helpers: the comment-insensitive hash
that ties the ncu traffic record to the kernel sources, the clock summary
over the timed window, and the credit width of each lifting launch that the
algorithmic bytes are priced at."""
from __future__ import annotations

import json
import os

import bench


def test_strip_comments_keeps_code_and_literals():
    src = 'int a = 1; // note\n/* block\n */ const char *s = "a//b /* q */"; char c = \'/\'; char e = \'\\\'\';\n'
    out = bench.strip_comments(src)
    assert "note" not in out and "block" not in out
    assert '"a//b /* q */"' in out and "'/'" in out and "'\\''" in out
    assert "int a = 1;" in out


def test_comment_edit_keeps_the_hash_code_edit_changes_it():
    code = "__global__ void k(int *p) { p[0] = 1; }\n"
    h1 = bench.strip_comments("// first version\n" + code)
    h2 = bench.strip_comments("/* reworded */\n" + code)
    assert h1.strip() == h2.strip()
    assert bench.strip_comments(code.replace("= 1", "= 2")) != bench.strip_comments(code)
    # comment lines leave blank lines behind; the hash collapses whitespace
    norm = lambda x: " ".join(bench.strip_comments(x).split())
    assert norm("// a\n// b\n// c\n" + code) == norm(code)


def test_traffic_records_name_a_kernel_hash_and_bytes():
    for name, key in (("fixpoint_grid4000_traffic.json", "dram_bytes_per_solve"),
                      ("fixpoint_rmat20_traffic.json", "dram_bytes_per_solve")):
        rec = json.load(open(os.path.join(bench.ROOT, "profiles", name)))
        assert rec[key] == rec["dram_bytes_read"] + rec["dram_bytes_write"] > 0
        assert len(rec["kernel_source_sha256"]) == 64
        assert rec["command"].startswith("ncu ") and "--clock-control none" in rec["command"]



def test_clock_summary_prefers_samples_inside_the_timed_window():
    clk = bench.ClockSampler(0)
    row = lambda mhz, slow="Not Active": ["0", str(mhz), "2070", "900", "0x0", slow, "Not Active", "Not Active",
                                          "Not Active"]
    clk.rows = [(1.0, row(1000)), (2.0, row(2070)), (2.01, row(2060, "Active")), (5.0, row(500))]
    clk.t0, clk.t1 = 1.9, 2.02
    s = clk.summary()
    assert s["window"] == "timed" and s["samples"] == 2 and s["sm_mhz"] == 2065
    assert s["reasons"] == ["hw_slowdown"]
    clk.t0, clk.t1 = 3.0, 3.01  # nothing inside: fall back to every sample
    s = clk.summary()
    assert s["window"] == "warm-up and timed" and s["samples"] == 4


def _phase(kind, cap, relax):
    return {"kind": kind, "cap": cap, "rounds": 1, "relaxations": relax, "ms": 1.0}


def test_lift_widths_follow_the_int32_rule():
    # config 3's route: int64 solve, every trial lift narrow (caps 4000 / 20000, 16000 / 528000)
    st = {"credit_bits": 64, "phase_list": [_phase("capped", 4000, 10), _phase("dual", 20000, 10),
                                            _phase("capped", 16000, 10), _phase("dual", 528000, 10)]}
    assert bench.lift_widths(st, 1000) == [32, 32, 32, 32]
    assert bench.credit_bytes(st, 1000) == 4.0
    # weights x 1e5: the capped lifts fit (4e8 + 1e8), the dual (K = 4) does not (2e9 + 4e8 + 1)
    B = 4 * 10**8
    st = {"credit_bits": 64, "phase_list": [_phase("attempt", 10**15, 30), _phase("capped", B, 10),
                                            _phase("dual", 5 * B, 20)]}
    assert bench.lift_widths(st, 10**8) == [64, 32, 64]
    assert bench.credit_bytes(st, 10**8) == (30 * 64 + 10 * 32 + 20 * 64) / 60 / 8
    # exactly at the limit: cap + |w| = 2^31 - 2 still fits below TOP = 2^31 - 1
    st = {"credit_bits": 64, "phase_list": [_phase("capped", 2**31 - 2 - 1000, 1)]}
    assert bench.lift_widths(st, 1000) == [32]
    st["phase_list"][0]["cap"] += 1
    assert bench.lift_widths(st, 1000) == [64]
    # an int32 solve: every launch int32; no phases: the solve's width
    assert bench.lift_widths({"credit_bits": 32, "phase_list": [_phase("attempt", 10**6, 5)]}, 100) == [32]
    assert bench.credit_bytes({"credit_bits": 64, "phase_list": []}, 100) == 8.0
