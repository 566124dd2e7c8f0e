"""Host logic of bench.py (no GPU): the clock record parsed from nvidia-smi samples, and the
DRAM traffic record tied to the rebuild kernel's source."""
import bench


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


def test_traffic_record_tied_to_the_kernel_source():
    # the committed record of the prefractured block was taken on the current rebuild source
    assert bench.traffic_from_profile("prefractured_block") == 412_581_632.0
    assert bench.traffic_from_profile("no_such_workload") is None
