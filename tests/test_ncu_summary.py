"""Host logic of the profile summaries (no GPU, no ncu run): the launch-list table of an
`ncu --metrics gpu__time_duration.sum --csv` log."""
import ncu_summary as N

CSV = '''==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python","h","void sta::(anonymous namespace)::k_fold_flat<4, false>(sta::FoldArgs, const int4 *, long, sta::(anonymous namespace)::FxArgs)","1","7","(128, 1, 1)","(1216, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ns","120,000"
"1","1","python","h","void sta::(anonymous namespace)::k_fold_flat<4, false>(sta::FoldArgs, const int4 *, long, sta::(anonymous namespace)::FxArgs)","1","7","(128, 1, 1)","(1216, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","usecond","80"
"2","1","python","h","void at::native::vectorized_elementwise_kernel<4, at::native::FillFunctor<unsigned char>, std::array<char *, 1>>(int, at::native::FillFunctor<unsigned char>, std::array<char *, 1>)","1","7","(128, 1, 1)","(2048, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ms","0.05"
'''


def test_short_kernel_names():
    assert N.short("void sta::(anonymous namespace)::k_fold_flat<4, false>(sta::FoldArgs)") == \
        "k_fold_flat<4, false>"
    assert N.short("void at::native::vectorized_elementwise_kernel<4, at::native::FillFunctor"
                   "<unsigned char>>(int)") == "torch fill (L2 flush / zero)"


def test_launch_table_sums_and_shares_in_any_time_unit(tmp_path):
    f = tmp_path / "launches.csv"
    f.write_text(CSV)
    lines = N.launches(str(f)).splitlines()
    assert lines[0].split() == ["kernel", "launches", "total_ms", "share"]
    fold = next(l for l in lines if l.startswith("k_fold_flat"))
    fill = next(l for l in lines if l.startswith("torch fill"))
    # 120,000 ns + 80 us = 0.200 ms; 0.05 ms of fill: shares 80% and 20%
    assert fold.split()[-3:] == ["2", "0.200", "80.0%"]
    assert fill.split()[-3:] == ["1", "0.050", "20.0%"]


def test_record_sums_the_launches_of_one_sequence(tmp_path, monkeypatch):
    hdr = ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum",
           "gpu__time_duration.sum"]
    units = ["", "", "Mbyte", "Kbyte", "usecond"]
    rows = [["0", "void sta::(anonymous namespace)::k_tile_flags(const unsigned char *)", "10", "200", "40"],
            ["1", "void sta::(anonymous namespace)::k_fold_flat<4, 0, 1>(sta::FoldArgs)", "150", "24,000", "60"],
            ["2", "void sta::(anonymous namespace)::k_stream_claim(const int *)", "1", "1", "9"]]
    monkeypatch.setattr(N, "_raw", lambda rep: (hdr, units, rows))
    out = tmp_path / "rebuild_wl.json"
    rec = N.record("x.ncu-rep", "rebuild", "wl", str(out), "k_fold_flat|k_tile_flags")
    assert rec["kernels"] == ["k_tile_flags", "k_fold_flat<4, 0, 1>"]
    assert rec["dram_bytes_read"] == 160e6 and rec["dram_bytes_write"] == 200e3 + 24e6
    assert rec["duration_us_cold"] == 100.0
    assert rec["source_sha"] == N.source_sha("rebuild") and out.exists()
    assert N.current_record("rebuild", "wl", tmp_path)["dram_bytes_per_launch"] == 160e6 + 24.2e6


def test_record_hash_ignores_comments_only():
    code = "int f(int x) {\n    return x + 1;  // one more\n}\n"
    assert N.code_of(code) == N.code_of("/* a\n note */\nint f(int x) {\n\n    return x + 1;\n}\n")
    assert N.code_of(code) != N.code_of(code.replace("x + 1", "x + 2"))
