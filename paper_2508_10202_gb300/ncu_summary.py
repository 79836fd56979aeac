"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel.

Usage: python -m paper_2508_10202_gb300.ncu_summary <launches.csv> [n_setup_launches]
The first n_setup_launches launches (one-time operator setup) are reported
apart from the matvec launches.  Prints a markdown table: launches, total
time, mean time and share per kernel.
"""
import collections
import csv
import re
import sys


def main(path, n_setup=0):
    rows = list(csv.reader(open(path)))
    start = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    hdr = rows[start]
    ki, mi, vi, ui = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    scale = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0}
    launches = []
    for r in rows[start + 1:]:
        if len(r) > vi and r[mi] == "gpu__time_duration.sum":
            name = re.sub(r"\(.*", "", r[ki].replace("(anonymous namespace)::", ""))
            name = name.replace("fftmv::<unnamed>::", "").replace("unnamed>::", "").replace("fftmv::", "")
            launches.append((name, float(r[vi].replace(",", "")) * scale[r[ui]]))
    for title, part in (("setup", launches[:n_setup]), ("matvec", launches[n_setup:])):
        agg = collections.OrderedDict()
        for n, t in part:
            a = agg.setdefault(n, [0, 0.0])
            a[0] += 1
            a[1] += t
        tot = sum(a[1] for a in agg.values()) or 1.0
        print(f"\n{title} launches: {len(part)}, {tot:.3f} ms\n")
        print("| kernel | launches | total ms | mean ms | share |\n|---|---|---|---|---|")
        for n, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
            print(f"| `{n}` | {c} | {t:.3f} | {t / c:.4f} | {100 * t / tot:.1f} % |")


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 0)
