"""Summaries of Nsight Compute output for this library's kernels (text for profiles/).

    python -m paper_2605_11673_gb300.ncu_summary launches <launches.csv>
        per kernel of an `ncu --metrics gpu__time_duration.sum --csv` launch list: launches,
        total device time, share (ncu's per-launch times are cold-cache and serialised, so
        compare shares, not absolutes)
    python -m paper_2605_11673_gb300.ncu_summary full <report.ncu-rep>
        key counters of every captured launch of an `ncu --set full` report
    python -m paper_2605_11673_gb300.ncu_summary traffic <report.ncu-rep> <kernel regex> \
            <workload> <out.json> [command]
        DRAM bytes per launch of the first matching launch, recorded with the hash of the
        rebuild kernel's source (bench.py reports the traffic only while that hash matches)
    python -m paper_2605_11673_gb300.ncu_summary run <prefractured|refinement> [--stream] [--proxy]
        the program to capture: one context on the workload (--proxy: the graph-Laplacian
        proxy operator), sta_full_rebuild of the initial mask, 3 sta_refold calls after
        256 MiB L2 flushes, and (--stream) the 24-frame edit stream through sta_apply_edits
        without CUDA graphs, each frame after a flush
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

CSRC = Path(__file__).resolve().parent / "csrc"
# the sources the rebuild kernel is compiled from (its traffic record is tied to them)
REBUILD_SOURCES = ("sta_rebuild.cu", "sta_fold.cuh")

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


def rebuild_source_sha() -> str:
    h = hashlib.sha256()
    for name in REBUILD_SOURCES:
        h.update((CSRC / name).read_bytes())
    return h.hexdigest()[:16]


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


def _bytes(value: str, unit: str) -> float:
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}[unit]
    return float(value.replace(",", "")) * scale


def traffic(rep: str, kernel: str, workload: str, out_json: str, command: str = "") -> dict:
    hdr, units, rows = _raw(rep)
    ki = hdr.index("Kernel Name")
    r = next(r for r in rows if re.search(kernel, r[ki]))
    col = {k: hdr.index(k) for k in ("dram__bytes_read.sum", "dram__bytes_write.sum",
                                      "gpu__time_duration.sum")}
    rd = _bytes(r[col["dram__bytes_read.sum"]], units[col["dram__bytes_read.sum"]])
    wr = _bytes(r[col["dram__bytes_write.sum"]], units[col["dram__bytes_write.sum"]])
    t = float(r[col["gpu__time_duration.sum"]].replace(",", ""))
    t_us = t * NS_PER.get(units[col["gpu__time_duration.sum"]], 1e3) / 1e3
    rec = {"kernel": short(r[ki]), "workload": workload, "source_sha": rebuild_source_sha(),
           "sources": list(REBUILD_SOURCES), "dram_bytes_read": rd, "dram_bytes_write": wr,
           "dram_bytes_per_launch": rd + wr, "duration_us_cold": t_us, "command": command}
    Path(out_json).write_text(json.dumps(rec, indent=1) + "\n")
    return rec


def run(workload: str, stream: bool = False, proxy: bool = False) -> None:
    import torch
    import paper_2605_11673_gb300 as P
    sys.path.insert(0, str(Path(__file__).resolve().parent.parent))
    import workloads as W
    wl = {"prefractured": W.prefractured_block, "refinement": W.refinement_hierarchy}[workload]()
    asm = (P.ProxyAssembler(wl.n_nodes, wl.tets, eps=1e-3) if proxy
           else P.Assembler(wl.X, wl.tets, wl.E, wl.nu))
    asm.full_rebuild(wl.mask0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        flush.zero_()
        asm.refold()
    if stream:
        for ed in wl.frames:
            flush.zero_()
            asm.apply_edits(ed)
    torch.cuda.synchronize()
    print("ok", workload, asm.sizes())
    asm.close()


if __name__ == "__main__":
    cmd, args = sys.argv[1], sys.argv[2:]
    if cmd == "run":
        run(args[0], "--stream" in args, "--proxy" in args)
    elif cmd == "launches":
        print(launches(args[0]))
    elif cmd == "full":
        print(full(args[0]))
    elif cmd == "traffic":
        print(json.dumps(traffic(*args), indent=1))
    else:
        raise SystemExit(__doc__)
