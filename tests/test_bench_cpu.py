"""Host-side logic of bench.py (no GPU): the clock-record summary and its
throttle flags, the kernel hash that ties the committed traffic record to
the kernel source, and the traffic lookup."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    return c.summary()


def test_clock_summary_median_and_reasons():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1995, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _sampler(lines)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_skips_garbage():
    lines = ["garbage", "",
             "0, 1500, 2070, 1400.0, 0x40, Active, Active, Not Active, Not Active"]
    s = _sampler(lines)
    assert s["samples"] == 1 and s["sm_mhz"] == 1500.0
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = _sampler([])
    assert s["samples"] == 0 and s["reasons"] == ["unsampled"]


def test_kernel_hash_ignores_comments_only(tmp_path, monkeypatch):
    """A comment or blank-space edit keeps the hash; a code edit changes it."""
    files = []
    for p in bench.KERNEL_SRCS:
        q = tmp_path / os.path.basename(p)
        shutil.copy(p, q)
        files.append(str(q))
    monkeypatch.setattr(bench, "KERNEL_SRCS", files)
    h0 = bench.kernel_hash()
    src = open(files[0]).read()
    open(files[0], "w").write("// a new comment\n" + src.replace("\n", "\n\n", 3) + "\n/* end */\n")
    assert bench.kernel_hash() == h0
    open(files[0], "w").write(src + "\nstatic int one_more_line = 1;\n")
    assert bench.kernel_hash() != h0


def test_traffic_lookup_needs_matching_hash(monkeypatch):
    """The traffic record is used only while its kernel hash matches."""
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0000000000000000")
    assert bench.ncu_traffic("k_step", "fp32", "5x512x512") is None


def test_replica_throughput_is_weak_scaling():
    assert bench.replica_throughput(100.0, 4, 2.0) == pytest.approx(200.0)


def test_traffic_record_is_for_this_kernel_source():
    """The DRAM traffic the bench reports comes from profiles/traffic.json,
    taken with ncu on a given kernel source: every entry must carry the
    current source's hash (else the bench reports traffic null and the
    profiles describe another kernel)."""
    import json
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    assert rec, "no traffic record"
    h = bench.kernel_hash()
    for key, e in rec.items():
        assert e["kernel_sha"] == h, key
        assert e["dram_bytes_per_launch"] > 0
    assert bench.ncu_traffic("k_step", "fp32", "5x512x512") == rec["k_step:fp32:5x512x512"]["dram_bytes_per_launch"]
