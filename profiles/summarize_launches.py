"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) by kernel: launches,
total device time and share.  Usage: python profiles/summarize_launches.py launches.csv"""
import collections
import csv
import io
import re
import sys


def summarize(path):
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    rows = list(csv.DictReader(io.StringIO("".join(lines))))
    agg = collections.OrderedDict()
    for r in rows:
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = re.sub(r"\(.*", "", r["Kernel Name"]).replace("(anonymous namespace)::", "")
        m = re.search(r"csr_rows<(\d+), (\w+), (\d)>", r["Kernel Name"])
        if m:
            name = f"csr_rows<{m.group(1)},{m.group(2)},{['spmv','residual','cheb','add'][int(m.group(3))]}>"
        v = float(r["Metric Value"])
        if r["Metric Unit"] in ("usecond", "us"):
            v *= 1e3
        elif r["Metric Unit"] in ("msecond", "ms"):
            v *= 1e6
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += v
    tot = sum(a[1] for a in agg.values())
    out = [f"{'launches':>8} {'total_ms':>10} {'share':>7}  kernel", "-" * 70]
    for k, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append(f"{c:8d} {t / 1e6:10.3f} {100 * t / tot:6.2f}%  {k}")
    out.append(f"{sum(a[0] for a in agg.values()):8d} {tot / 1e6:10.3f} 100.00%  (all)")
    return "\n".join(out)


if __name__ == "__main__":
    print(summarize(sys.argv[1]))
