"""Summarise an ncu --csv launch list (gpu__time_duration.sum per launch) by kernel:
launches, total time and share.  Usage: python launch_summary.py launches.csv [--exclude name,...]
(excluded kernels, e.g. the benchmark's L2 flush fill and its timed spin, are left out of
the shares)."""
import collections
import csv
import re
import sys


def summarise(path, exclude=()):
    rows = list(csv.reader(open(path)))
    start = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[start]
    ki, mi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    agg = collections.OrderedDict()
    scale = {"nsecond": 1.0, "ns": 1.0, "usecond": 1e3, "us": 1e3, "msecond": 1e6, "ms": 1e6}
    for r in rows[start + 1:]:
        if len(r) <= mi:
            continue
        name = re.sub(r"^void ", "", r[ki].split("(")[0])
        name = re.sub(r"<.*", "", name.replace("<unnamed>", "anon")).split("::")[-1]
        if name in exclude:
            continue
        v = float(r[mi].replace(",", "")) * scale.get(r[ui], 1.0)
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += v
    tot = sum(a[1] for a in agg.values())
    lines = ["%-34s %8s %12s %7s" % ("kernel", "launches", "total_us", "share")]
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        lines.append("%-34s %8d %12.1f %6.1f%%" % (k, n, t / 1e3, 100 * t / tot))
    return "\n".join(lines)


if __name__ == "__main__":
    ex = ()
    if "--exclude" in sys.argv:
        ex = tuple(sys.argv[sys.argv.index("--exclude") + 1].split(","))
    print(summarise(sys.argv[1], ex))
