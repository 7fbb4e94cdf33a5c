"""Summarise an ncu launch list (``--metrics gpu__time_duration.sum --csv``) per kernel.

Usage: python -m paper_2508_18468_gb300.profiling <launches.csv>
Prints launches, total time and share of every kernel, largest first.
"""
import collections
import csv
import re
import sys

SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3,
         "second": 1e3}


def main(path):
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, mi, vi, ui = (hdr.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    tot, cnt = collections.defaultdict(float), collections.Counter()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = re.sub(r"\(CUtensorMap.*|\((const |int|long|float|double|cplx|__half|unsigned).*", "", r[ki]).strip()
        tot[name] += float(r[vi].replace(",", "")) * SCALE[r[ui]]
        cnt[name] += 1
    T = sum(tot.values())
    print("launches %d, total %.1f ms" % (sum(cnt.values()), T))
    print("%8s %12s %7s  %s" % ("launches", "total ms", "share", "kernel"))
    for k, v in sorted(tot.items(), key=lambda x: -x[1]):
        print("%8d %12.2f %6.1f%%  %s" % (cnt[k], v, 100 * v / T, k))


if __name__ == "__main__":
    main(sys.argv[1])
