"""Summarise an ncu --csv launch list (gpu__time_duration.sum) per kernel:
launches, total time and share.  Usage: python summarize_launches.py launches.csv"""
import collections
import csv
import sys

rows = list(csv.reader(open(sys.argv[1])))
hi = [i for i, r in enumerate(rows) if "Kernel Name" in r][0]
h = rows[hi]
ki, mi, vi, ui = (h.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}
agg = collections.defaultdict(lambda: [0, 0.0])
for r in rows[hi + 1:]:
    if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
        continue
    us = float(r[vi].replace(",", "")) * scale[r[ui]]
    name = r[ki].split("(")[0]
    agg[name][0] += 1
    agg[name][1] += us
tot = sum(v[1] for v in agg.values())
print(f"{'launches':>8} {'total ms':>10} {'share':>7}  kernel")
for k, v in sorted(agg.items(), key=lambda x: -x[1][1]):
    print(f"{v[0]:8d} {v[1] / 1e3:10.3f} {100 * v[1] / tot:6.2f}%  {k}")
