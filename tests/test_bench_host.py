"""Host logic of bench.py (no GPU): the clock record parsed from nvidia-smi samples, and the
ncu records (DRAM traffic, FP64 instructions per tet) used only while they match the current
sources of their kernel."""
import json

import bench
import ncu_summary


def test_clock_samples_parse():
    out = "\n".join([
        "2070, 2070, 612.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 990.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "[N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "garbage",
        "1995, 2070, 1300.5, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
    ])
    rec = bench.ClockSampler.parse(out)
    assert rec == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0,
                   "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}
    assert bench.ClockSampler.parse("") is None
    assert bench.ClockSampler.parse("n/a, n/a, n/a, n/a, a, b, c, d") is None


def _write_record(d, kernel, workload, sha, **extra):
    rec = dict({"kernel": kernel, "workload": workload, "source_sha": sha}, **extra)
    (d / f"{kernel}_{workload}.json").write_text(json.dumps(rec))


def test_records_used_only_on_the_current_kernel_source(tmp_path):
    cur = ncu_summary.source_sha("rebuild")
    _write_record(tmp_path, "rebuild", "wl", cur, dram_bytes_per_launch=123.0)
    _write_record(tmp_path, "rebuild", "old", "0" * 16, dram_bytes_per_launch=456.0)
    assert bench.traffic_from_profile("wl", tmp_path) == 123.0
    assert bench.traffic_from_profile("old", tmp_path) is None  # stale hash
    assert bench.traffic_from_profile("missing", tmp_path) is None
    _write_record(tmp_path, "k_elements", "wl", ncu_summary.source_sha("k_elements"),
                  fp64_inst_per_unit=300.0)
    _write_record(tmp_path, "k_adjoint", "wl", "f" * 16, fp64_inst_per_unit=900.0)
    assert bench.fp64_per_tet("k_elements", "wl", tmp_path) == 300.0
    assert bench.fp64_per_tet("k_adjoint", "wl", tmp_path) is None


def test_source_hash_covers_the_kernel_and_its_layout():
    # the rebuild's traffic depends on the unit order that create builds
    assert "sta_create.cu" in ncu_summary.KERNEL_SOURCES["rebuild"]
    for k, srcs in ncu_summary.KERNEL_SOURCES.items():
        assert all((ncu_summary.CSRC / f).exists() for f in srcs), k
    assert ncu_summary.source_sha("k_elements") != ncu_summary.source_sha("rebuild")
