"""bench.py's host-side helpers on the CPU: the clock record's parsing, the
kernel-source hash that ties a committed ncu capture to the sources, and the
traffic figure read from that capture."""
import os
import shutil

import pytest

import bench


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return "0, %s, %s, 900.0, 0x0, %s, %s, %s, %s" % (sm, mx, hw, hwt, swt, cap)


def test_clock_summary_median_max_and_reasons():
    c = bench.ClockSampler(0)
    c.lines = [_line(2070, 2070), _line(1980, 2070, cap="Active"), _line(2040, 2070), "garbage", ""]
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = [_line(1200, 2070, hw="Active", swt="Active")]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_kernel_hash_ignores_comments_and_other_sections_not_pair_code(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_0909_5215_gb300", "csrc")
    dst = tmp_path / "paper_0909_5215_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("hd_kernels.cu", "hd_internal.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_code_hash()
    k = dst / "hd_kernels.cu"
    k.write_text(k.read_text() + "\n// a comment\n/* and a\n   block comment */\n\n")
    assert bench.kernel_code_hash() == h0
    k.write_text(k.read_text() + "\nstatic int extra_symbol_outside_the_pair_sweep;\n")
    assert bench.kernel_code_hash() == h0            # the launchers section is not the pair kernel's
    text = k.read_text()
    red = text.index("// ---------------------------------------------------------------- reductions")
    at = text.index("\n", red) + 1
    k.write_text(text[:at] + "static int extra_symbol_in_the_reductions;\n" + text[at:])
    assert bench.kernel_code_hash() != h0
    k.write_text(text)
    assert bench.kernel_code_hash() == h0
    mark = text.index("// ---------------------------------------------------------------- pair sweep")
    at = text.index("\n", mark) + 1
    k.write_text(text[:at] + "static int extra_symbol_in_the_pair_sweep;\n" + text[at:])
    assert bench.kernel_code_hash() != h0


def test_committed_traffic_is_tied_to_the_sources(monkeypatch):
    assert bench.committed_traffic(False) is None
    t = bench.committed_traffic(True)
    text = open(os.path.join(bench.ROOT, "profiles", "k_pair32_afm3d_hyper64.md")).read()
    kv = dict(l.split(": ", 1) for l in text.splitlines() if l.startswith(("traffic_bytes", "kernel_code")))
    if bench.kernel_code_hash() == kv["kernel_code_sha256_16"].strip():
        assert t == float(kv["traffic_bytes_per_launch"])
    else:
        assert t is None
    monkeypatch.setattr(bench, "kernel_code_hash", lambda: "0" * 16)
    assert bench.committed_traffic(True) is None


def test_quench_summary_reports_the_three_outcomes():
    import argparse
    args = argparse.Namespace(quench_ftol=1e-2, quench_stay=1e-1, quench_iters=3000)
    qs = [{"iters": 400.0, "iters_max": 1200, "converged": 0.1, "stayed": 0.9, "fmax": 0.009, "fmax_stay": 0.09,
           "fmax_unconverged": 0.0, "flagged": 1},
          {"iters": 500.0, "iters_max": 3000, "converged": 0.0, "stayed": 0.8, "fmax": 0.0, "fmax_stay": 0.095,
           "fmax_unconverged": 0.5, "flagged": 0}]
    s = bench.quench_summary(qs, args, ms=100.0, md_ms=60.0, seed={"converged": 2, "of": 2})
    assert s["iters_mean"] == pytest.approx(450.0) and s["iters_max"] == 3000
    assert s["converged_fraction"] == pytest.approx(0.05) and s["stayed_fraction"] == pytest.approx(0.85)
    assert s["unconverged_fraction"] == pytest.approx(0.10)
    assert s["fmax_max_converged"] == 0.009 and s["fmax_max_stayed"] == 0.095 and s["fmax_max_unconverged"] == 0.5
    assert s["flagged"] == 1 and s["time_share"] == pytest.approx(0.4) and s["ftol_stay"] == 1e-1
