"""Summarise an ncu CSV launch list (``--metrics gpu__time_duration.sum --csv``)
per kernel: launches, total device time and share.  Usage:

    python -m paper_2511_16174_gb300.ncu_summary launches.csv [--only evd::] [--md]
"""
from __future__ import annotations

import csv
import re
import sys
from collections import defaultdict


def summarize(path, only=None):
    rows = []
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    rd = csv.DictReader(lines)
    agg = defaultdict(lambda: [0, 0.0])
    for r in rd:
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = r["Kernel Name"]
        short = re.sub(r"\(.*", "", name)
        short = re.sub(r"evd::(\(anonymous namespace\)|_GLOBAL__N_\w+)::", "evd::", short)
        if only and only not in short:
            continue
        t = float(r["Metric Value"].replace(",", ""))
        unit = r.get("Metric Unit", "ns")
        if unit == "us":
            t *= 1e3
        elif unit == "ms":
            t *= 1e6
        agg[short][0] += 1
        agg[short][1] += t
    total = sum(v[1] for v in agg.values())
    out = sorted(agg.items(), key=lambda kv: -kv[1][1])
    return [(k, v[0], v[1] / 1e6, v[1] / total if total else 0.0) for k, v in out], total / 1e6


def main():
    path = sys.argv[1]
    only = None
    if "--only" in sys.argv:
        only = sys.argv[sys.argv.index("--only") + 1]
    rows, total = summarize(path, only)
    print("| kernel | launches | total ms | share |")
    print("|---|---:|---:|---:|")
    for k, n, ms, sh in rows:
        print(f"| `{k}` | {n} | {ms:.2f} | {100 * sh:.1f}% |")
    print(f"| total | {sum(r[1] for r in rows)} | {total:.2f} | 100% |")


if __name__ == "__main__":
    main()
