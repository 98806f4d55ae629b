"""Summarise an ncu --csv launch list (metric gpu__time_duration.sum) per
kernel: launches, total time and share of the total.

Usage: python -m paper_0909_5257_gb300.ncu_launches launches.csv"""
import collections
import csv
import sys

_SCALE_US = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}


def summarize(path):
    """Return [(kernel, launches, total_ms, share)] sorted by total time."""
    rows = list(csv.reader(open(path)))
    hi = [i for i, r in enumerate(rows) if "Kernel Name" in r][0]
    h = rows[hi]
    ki, mi, vi, ui = (h.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        us = float(r[vi].replace(",", "")) * _SCALE_US[r[ui]]
        name = r[ki].split("(")[0]
        agg[name][0] += 1
        agg[name][1] += us
    tot = sum(v[1] for v in agg.values()) or 1.0
    return [(k, v[0], v[1] / 1e3, v[1] / tot) for k, v in sorted(agg.items(), key=lambda x: -x[1][1])]


def main(argv):
    print(f"{'launches':>8} {'total ms':>10} {'share':>7}  kernel")
    for k, n, ms, share in summarize(argv[1]):
        print(f"{n:8d} {ms:10.3f} {100 * share:6.2f}%  {k}")


if __name__ == "__main__":
    main(sys.argv)
