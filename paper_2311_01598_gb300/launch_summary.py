"""Summarise an ncu launch list (gpu__time_duration.sum per launch) by kernel.

The library counts its own launches (ks_kernel_launches); bench.py reports
the counter value at the start of its timed region and the number of
launches inside it ("launch_window").  Given the CSV of
`ncu --metrics gpu__time_duration.sum --csv --log-file …` over the same
command and that window, this prints per kernel its launches, total time
and share of the window, as a markdown table.  Library kernels are the ones
named k_*; other launches (PyTorch's) are ignored.

    python -m paper_2311_01598_gb300.launch_summary launches.csv --first F --count C
"""
from __future__ import annotations

import argparse
import csv
import json
import re


def read_launches(path):
    """[(kernel_name, grid, ns)] of the library's launches in launch order."""
    rows = []
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = r["Kernel Name"]
        m = re.match(r"(?:void )?(k_[A-Za-z0-9_]+(?:<[^()]*>)?)", name)
        if not m:
            continue
        ns = float(r["Metric Value"].replace(",", ""))
        if r.get("Metric Unit") == "us":
            ns *= 1e3
        elif r.get("Metric Unit") == "ms":
            ns *= 1e6
        rows.append((m.group(1), r["Grid Size"], ns))
    return rows


def summarise(rows, first, count):
    win = rows[first:first + count] if count else rows[first:]
    per = {}
    for name, _, ns in win:
        c, t = per.get(name, (0, 0.0))
        per[name] = (c + 1, t + ns)
    total = sum(t for _, t in per.values())
    table = sorted(((n, c, t, t / total if total else 0.0) for n, (c, t) in per.items()), key=lambda x: -x[2])
    return table, total, len(win)


def to_markdown(table, total, n):
    out = [f"{n} launches, {total / 1e3:.1f} us total (ncu: cold cache, serialised)", "",
           "| kernel | launches | total us | share |", "|---|---|---|---|"]
    for name, c, t, sh in table:
        out.append(f"| `{name}` | {c} | {t / 1e3:.1f} | {100 * sh:.1f}% |")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--count", type=int, default=0)
    ap.add_argument("--bench-json", default=None,
                    help="bench.py output; its launch_window replaces --first/--count")
    a = ap.parse_args()
    first, count = a.first, a.count
    if a.bench_json:
        with open(a.bench_json) as f:
            line = [ln for ln in f if ln.startswith("{")][-1]
        w = json.loads(line)["launch_window"]
        first, count = w["first"], w["count"]
    rows = read_launches(a.csv)
    table, total, n = summarise(rows, first, count)
    print(to_markdown(table, total, n))


if __name__ == "__main__":
    main()
