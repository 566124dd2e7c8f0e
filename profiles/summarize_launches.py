"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel:
launches, total device time and share.  Usage: python profiles/summarize_launches.py <csv>"""
import collections
import csv
import re
import sys


def short(name: str) -> str:
    m = re.search(r"\b(k_\w+)(<[^>(]*>)?", name)
    if m:
        return m.group(1) + (m.group(2) or "")
    if "FillFunctor" in name:
        return "torch fill (L2 flush / zero)"
    return re.sub(r"\(.*", "", name)[:48]


def main(path):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, mi, vi = hdr.index("Kernel Name"), hdr.index("Metric Name"), hdr.index("Metric Value")
    tot = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hi + 1:]:
        if len(r) > vi and r[mi] == "gpu__time_duration.sum":
            k = short(r[ki])
            tot[k][0] += 1
            tot[k][1] += float(r[vi].replace(",", ""))
    total = sum(t for _, t in tot.values())
    print(f"{'kernel':44s} {'launches':>8s} {'total_ms':>9s} {'share':>7s}")
    for k, (n, t) in sorted(tot.items(), key=lambda kv: -kv[1][1]):
        print(f"{k:44s} {n:8d} {t / 1e6:9.3f} {100 * t / total:6.1f}%")


if __name__ == "__main__":
    main(sys.argv[1])
