"""The benchmark's contract pieces that run without a GPU: the reference arm's JSON line
(the FP64 oracle timed on the host cores), the clock-sample summary, and the lookup of
the committed DRAM-traffic record."""
import json
import os
import subprocess
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_line(orc):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["warmup"] >= 3  # the timing rule's minimum is enforced
    assert d["config"]["workload"] == "cfg2_3d_neumann_512"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_clock_summary_counts_only_samples_inside_the_region():
    c = bench.ClockSampler(0)
    c.t0 = time.time()
    row = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"
    c.lines = [(c.t0 - 1.0, row.format(sm=345, hw="Not Active", pc="Not Active")),  # before the region
               (c.t0 + 0.1, row.format(sm=2070, hw="Not Active", pc="Not Active")),
               (c.t0 + 0.2, row.format(sm=2055, hw="Not Active", pc="Active")),
               (c.t0 + 0.3, row.format(sm=2070, hw="Not Active", pc="Not Active")),
               (c.t0 + 0.4, "garbled")]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.lines.append((c.t0 + 0.5, row.format(sm=1500, hw="Active", pc="Not Active")))
    assert "hw_slowdown" in c.summary()["reasons"]
    empty = bench.ClockSampler(0)
    empty.t0 = time.time()
    assert empty.summary()["samples"] == 0


def test_traffic_record_lookup(tmp_path, monkeypatch):
    """The committed ncu traffic of a kernel is reported only while the digest of its
    sources matches the one recorded with the capture; an unknown tag gives none."""
    import hashlib
    src = tmp_path / "paper_2312_07010_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "a.cu").write_text("kernel a")
    (src / "b.cuh").write_text("header b")
    dig = hashlib.sha256(b"kernel a" + b"header b").hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(
        "# comment\n" f"k_tag a.cu,b.cuh 1038020480 {dig}\n" "k_old a.cu 5 0000000000000000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_from_profile("k_tag") == 1038020480.0
    assert bench._traffic_from_profile("k_old") is None
    assert bench._traffic_from_profile("no_such_kernel") is None
    (src / "a.cu").write_text("kernel a, changed")
    assert bench._traffic_from_profile("k_tag") is None
