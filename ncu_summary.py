"""Summaries of Nsight Compute output for this library's kernels (text for profiles/), and the
program those captures run.  Measurement tooling beside bench.py, not part of the library.

    python ncu_summary.py launches <launches.csv>
        per kernel of an `ncu --metrics gpu__time_duration.sum --csv` launch list: launches,
        total device time, share (ncu's per-launch times are cold-cache and serialised, so
        compare shares, not absolutes)
    python ncu_summary.py full <report.ncu-rep>
        key counters of every captured launch of an `ncu --set full` report
    python ncu_summary.py record <report.ncu-rep> <key> <workload> <out.json> \
            --kernels <regex> [--units N] [--command "..."]
        counters summed over the captured launches of the kernels matching <regex> -- one
        launch sequence, e.g. a rebuild's k_tile_flags + k_fold_flat (DRAM bytes, duration and,
        when captured, the FP64 thread instructions; --units: the work items it processed,
        e.g. active tetrahedra, for per-unit figures) -- recorded as <key>_<workload> with the
        hash of the sources the kernels and their data layout are built from
        (KERNEL_SOURCES[key]): bench.py uses a record only while that hash matches
    python ncu_summary.py run <workload> [--stream] [--proxy] [--elements]
        the program to capture: one context on the workload (prefractured, refinement,
        refinement_r040; --proxy: the graph-Laplacian proxy operator), sta_full_rebuild of
        the initial mask, 3 sta_refold calls after 256 MiB L2 flushes, (--elements) the
        element kernel over the active tetrahedra and the adjoint kernel for a seeded
        gradient, 2 launches each after a flush, and (--stream) the 24-frame edit stream
        through sta_apply_edits without CUDA graphs, each frame after a flush
"""
from __future__ import annotations

import collections
import csv
import hashlib
import json
import re
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parent
CSRC = ROOT / "paper_2605_11673_gb300" / "csrc"
# the sources each recorded kernel and the data layout it reads are built from: a record is
# current only while these hash to the value it was taken with (the rebuild's traffic also
# depends on the unit order and tiles that create builds)
KERNEL_SOURCES = {
    "rebuild": ("sta_rebuild.cu", "sta_fold.cuh", "sta_create.cu", "sta_internal.cuh"),
    "k_elements": ("sta_element.cu", "sta_internal.cuh"),
    "k_adjoint": ("sta_element.cu", "sta_internal.cuh"),
}
# FP64 thread instructions (predicated on), when a capture collected them
FP64_INST = ("smsp__sass_thread_inst_executed_op_dadd_pred_on.sum",
             "smsp__sass_thread_inst_executed_op_dmul_pred_on.sum",
             "smsp__sass_thread_inst_executed_op_dfma_pred_on.sum")

KEYS = ["gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
        "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "launch__grid_size",
        "launch__block_size", "launch__registers_per_thread",
        "sm__warps_active.avg.pct_of_peak_sustained_active",
        "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active",
        "smsp__inst_executed.sum",
        "smsp__thread_inst_executed_per_inst_executed.ratio",
        "smsp__issue_active.avg.pct_of_peak_sustained_active",
        "lts__t_sector_hit_rate.pct", "l1tex__t_sector_hit_rate.pct",
        "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio",
        "smsp__average_warps_issue_stalled_wait_per_issue_active.ratio",
        "smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio",
        "smsp__average_warps_issue_stalled_math_pipe_throttle_per_issue_active.ratio"]


def code_of(text: str) -> str:
    """C/CUDA source without its comments, trailing blanks and empty lines: what the compiler
    sees, so that a record stays current through a comment-only edit."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def source_sha(kernel: str) -> str:
    """Hash of the current code (comments left out) of the sources of a recorded kernel
    (KERNEL_SOURCES)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        h.update(code_of((CSRC / name).read_text()).encode())
    return h.hexdigest()[:16]


def current_record(kernel: str, workload: str, directory: Path | None = None):
    """The committed record profiles/<kernel>_<workload>.json if it was taken on the current
    sources of the kernel, else None."""
    p = Path(directory or ROOT / "profiles") / f"{kernel}_{workload}.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text())
    if d.get("source_sha") != source_sha(kernel):
        return None
    return d


def short(name: str) -> str:
    m = re.search(r"\b(k_\w+)(<[^>(]*>)?", name)
    if m:
        return m.group(1) + (m.group(2) or "")
    if "FillFunctor" in name:
        return "torch fill (L2 flush / zero)"
    return re.sub(r"\(.*", "", name)[:48]


# nanoseconds per time unit, in both spellings ncu prints (launch-list CSV, raw page)
NS_PER = {"ns": 1.0, "nsecond": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6,
          "s": 1e9, "second": 1e9}


def launches(path: str) -> str:
    with open(path) as fh:
        rows = list(csv.reader(fh))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, mi, vi = hdr.index("Kernel Name"), hdr.index("Metric Name"), hdr.index("Metric Value")
    ui = hdr.index("Metric Unit") if "Metric Unit" in hdr else None
    tot = collections.defaultdict(lambda: [0, 0.0])  # kernel -> [launches, total ns]
    for r in rows[hi + 1:]:
        if len(r) > vi and r[mi] == "gpu__time_duration.sum":
            k = short(r[ki])
            scale = NS_PER.get(r[ui], 1.0) if ui is not None else 1.0
            tot[k][0] += 1
            tot[k][1] += float(r[vi].replace(",", "")) * scale
    total = sum(t for _, t in tot.values())
    out = [f"{'kernel':44s} {'launches':>8s} {'total_ms':>9s} {'share':>7s}"]
    for k, (n, t) in sorted(tot.items(), key=lambda kv: -kv[1][1]):
        out.append(f"{k:44s} {n:8d} {t / 1e6:9.3f} {100 * t / total:6.1f}%")
    return "\n".join(out)


def _raw(rep: str):
    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True,
                         text=True, check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    return rows[0], rows[1], rows[2:]


def full(rep: str) -> str:
    hdr, units, rows = _raw(rep)
    idx = {k: hdr.index(k) for k in KEYS if k in hdr}
    out = []
    for r in rows:
        out.append(f"## {short(r[hdr.index('Kernel Name')])}")
        for k, i in idx.items():
            out.append(f"  {k} = {r[i]} {units[i]}")
    return "\n".join(out)


def _bytes(value, unit: str) -> float:
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}[unit]
    return float(str(value).replace(",", "")) * scale


def record(rep: str, key: str, workload: str, out_json: str, kernels: str, units: float = 0.0,
           command: str = "") -> dict:
    """Sum the counters of every captured launch whose kernel name matches `kernels` (the
    capture holds one launch sequence, e.g. the rebuild's k_tile_flags + k_fold_flat) and write
    the record <key>_<workload>.json, tied to the hash of KERNEL_SOURCES[key]."""
    hdr, unit_row, rows = _raw(rep)
    ki = hdr.index("Kernel Name")
    picked = [r for r in rows if re.search(kernels, short(r[ki]))]
    if not picked:
        raise SystemExit(f"no launch of {kernels!r} in {rep}")

    def val(r, name):
        i = hdr.index(name)
        return float(r[i].replace(",", "")), unit_row[i]

    rec = {"key": key, "kernels": [short(r[ki]) for r in picked], "workload": workload,
           "source_sha": source_sha(key), "sources": list(KERNEL_SOURCES[key])}
    rd = sum(_bytes(*val(r, "dram__bytes_read.sum")) for r in picked)
    wr = sum(_bytes(*val(r, "dram__bytes_write.sum")) for r in picked)
    t = sum(val(r, "gpu__time_duration.sum")[0] * NS_PER.get(val(r, "gpu__time_duration.sum")[1], 1e3)
            for r in picked) / 1e3
    rec.update({"dram_bytes_read": rd, "dram_bytes_write": wr, "dram_bytes_per_launch": rd + wr,
                "duration_us_cold": t})
    rec["per_kernel"] = {short(r[ki]): {
        "dram_bytes": _bytes(*val(r, "dram__bytes_read.sum")) + _bytes(*val(r, "dram__bytes_write.sum")),
        "duration_us_cold": val(r, "gpu__time_duration.sum")[0]
        * NS_PER.get(val(r, "gpu__time_duration.sum")[1], 1e3) / 1e3} for r in picked}
    if all(m in hdr for m in FP64_INST):
        fp64 = sum(val(r, m)[0] for r in picked for m in FP64_INST)
        rec["fp64_thread_inst"] = fp64
        for m in FP64_INST:
            rec[m] = sum(val(r, m)[0] for r in picked)
        if units:
            rec["units"] = units
            rec["fp64_inst_per_unit"] = fp64 / units
    for m in ("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active",
              "smsp__issue_active.avg.pct_of_peak_sustained_active",
              "smsp__inst_executed.sum"):
        if m in hdr:
            rec[m] = [val(r, m)[0] for r in picked]
    rec["command"] = command
    Path(out_json).write_text(json.dumps(rec, indent=1) + "\n")
    return rec


def run(workload: str, stream: bool = False, proxy: bool = False, elements: bool = False) -> None:
    import torch
    sys.path.insert(0, str(ROOT))
    import paper_2605_11673_gb300 as P
    import workloads as W
    wl = {"prefractured": W.prefractured_block, "refinement": W.refinement_hierarchy,
          "refinement_r040": lambda: W.refinement_hierarchy(radius=0.40)}[workload]()
    asm = (P.ProxyAssembler(wl.n_nodes, wl.tets, eps=1e-3) if proxy
           else P.Assembler(wl.X, wl.tets, wl.E, wl.nu))
    asm.full_rebuild(wl.mask0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        flush.zero_()
        asm.refold()
    if elements and not proxy:
        gen = torch.Generator(device="cuda").manual_seed(0)
        gval = torch.randn(asm.sizes()["nnz"], dtype=torch.float64, device="cuda", generator=gen)
        for _ in range(2):
            flush.zero_()
            asm.recompute_elements(active_only=True)
        for _ in range(2):
            flush.zero_()
            P.sta_adjoint(asm.h, gval)
    if stream:
        for ed in wl.frames:
            flush.zero_()
            asm.apply_edits(ed)
    torch.cuda.synchronize()
    print("ok", workload, asm.sizes(), "active", int(wl.mask0.sum()))
    asm.close()


def main(argv) -> None:
    import argparse
    ap = argparse.ArgumentParser(description="ncu summaries for profiles/")
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("run")
    a.add_argument("workload")
    a.add_argument("--stream", action="store_true")
    a.add_argument("--proxy", action="store_true")
    a.add_argument("--elements", action="store_true")
    sub.add_parser("launches").add_argument("csv")
    sub.add_parser("full").add_argument("report")
    a = sub.add_parser("record")
    for name in ("report", "key", "workload", "out_json"):
        a.add_argument(name)
    a.add_argument("--kernels", required=True, help="regex of the kernels to sum")
    a.add_argument("--units", type=float, default=0.0)
    a.add_argument("--command", default="")
    args = ap.parse_args(argv)
    if args.cmd == "run":
        run(args.workload, args.stream, args.proxy, args.elements)
    elif args.cmd == "launches":
        print(launches(args.csv))
    elif args.cmd == "full":
        print(full(args.report))
    else:
        print(json.dumps(record(args.report, args.key, args.workload, args.out_json,
                                args.kernels, args.units, args.command), indent=1))


if __name__ == "__main__":
    main(sys.argv[1:])
