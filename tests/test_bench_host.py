"""Host-side pieces of bench.py that need no GPU: the ncu figures it reports come from the
committed profile summary, both arms print the same workload description, and the FP32 ALU
peak is derived from the unit counts."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_ncu_figures_match_committed_profile():
    text = open(os.path.join(ROOT, bench.NCU_PROFILE)).read()
    table = text[text.index("Figures bench.py reports"):]
    rows = dict((m.group(1), (float(m.group(2)), None if m.group(3) == "-" else float(m.group(3))))
                for m in re.finditer(r"^\| (k_\S+) \| ([\d.]+) \| ([\d.]+|-) \|$", table, flags=re.M))
    for k, v in bench.NCU_WIDE.items():
        if v["traffic"] is None and v["tensor_pct"] is None:
            continue
        assert k in rows, k
        assert abs(rows[k][0] * 1e6 - v["traffic"]) < 0.05e6, (k, rows[k], v)
        if v["tensor_pct"] is None:
            assert rows[k][1] is None, (k, rows[k])
        else:
            assert abs(rows[k][1] - v["tensor_pct"]) < 0.05, (k, rows[k], v)


def test_both_arms_print_the_same_config():
    assert bench.config_dict(1) == bench.config_dict(1)
    c = bench.config_dict(1)
    assert c["m"] == c["n"] == 8192 and c["l"] == 120 and c["q"] == 2
    assert "8192x8192" in c["workload"]


def test_wide_phase_kernels_cover_the_roofline_candidates():
    for k in ("k_wd_pass<1,0>", "k_wd_pass<0,0>", "k_wd_alm<true>"):
        assert k in bench.WIDE_PHASE_KERNEL.values()
    assert 70.0 < bench.fp32_alu_peak_tflops() < 90.0
