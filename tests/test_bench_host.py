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


def test_wide_roofline_groups_from_phase_times():
    """The roofline groups computed from per-phase times: a pass's launch group is the pass with its
    partial sum, the sketch phase (Omega^T, then the first pass) is one unit of two launch groups,
    and the core group is reported against the FP32 issue rate."""
    K = 4
    ph = {"sketch": (0.100, 2), "power_AQ": (0.180, 2), "power_AtZ": (0.176, 2), "orth": (0.440, 4),
          "project": (0.090, 1), "core": (0.500, 1), "epilogue": (0.240, 1), "apply": (0.108, 5)}
    tm = {k: (ms * K, cnt * K) for k, (ms, cnt) in ph.items()}
    r = bench.wide_roofline(tm, K, 8192, 8)
    assert r["kernel"] == "k_wd_gram + k_wd_core" and r["bound"] == "alu"
    other = r["other_kernels"]
    e, z = 4.0 * 8192 * 8192, 4.0 * 128 * 8192
    peak, _ = bench.peaks()
    # sketch: 0.100 ms for one unit of e + 5 z bytes
    assert abs(other["k_wd_omega + k_wd_pass<1,0>"]["achieved"] - (e + 5 * z) / 0.100e-3 / 1e9) < 1e-6
    # row pass: (0.180 + 0.090) ms over 3 launch groups of e + 4 z bytes
    assert abs(other["k_wd_pass<0,0>"]["achieved"] - (e + 4 * z) / 0.090e-3 / 1e9) < 1e-6
    assert abs(other["k_wd_pass<1,0>"]["achieved"] - (e + 3 * z) / 0.088e-3 / 1e9) < 1e-6
    assert abs(other["k_wd_alm<true>"]["frac"] - (5 * e + 4 * z) / 0.240e-3 / 1e9 / peak) < 1e-9
    assert 0.0 < r["frac"] < 0.1
