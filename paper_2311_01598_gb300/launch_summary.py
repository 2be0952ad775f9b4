"""Summarise an ncu launch list (gpu__time_duration.sum per launch) by kernel.

The library counts its own launches (ks_kernel_launches); bench.py reports
the counter value at the start of its timed region and the number of
launches inside it ("launch_window").  Given the CSV of
`ncu --metrics gpu__time_duration.sum --csv --log-file …` over the same
command and that window, this prints per kernel its launches, total time
and share of the window, as a markdown table.  Library kernels are the ones
named k_* (namespace qualifiers allowed); other launches (PyTorch's) are
ignored.

    python -m paper_2311_01598_gb300.launch_summary launches.csv --first F --count C

`traffic` turns an ncu report of a few key switches into DRAM bytes per key
switch for each captured kernel and records them, with a hash of the kernel
sources they were taken on, in data/ncu_traffic_gb300.json (bench.py reports
them only while the sources are unchanged):

    python -m paper_2311_01598_gb300.launch_summary traffic prof.ncu-rep --key-switches 4 \
        --capture "<the ncu command>"

`pipes` records a kernel's integer-pipe utilisation (fmaheavy = the 32-bit
integer multiply pipe, ALU, issue) from an ncu report, the same way, in
data/ncu_pipes_gb300.json:

    python -m paper_2311_01598_gb300.launch_summary pipes prof.ncu-rep --capture "<the ncu command>"
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import re
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
TRAFFIC_PATH = os.path.join(HERE, "data", "ncu_traffic_gb300.json")
PIPES_PATH = os.path.join(HERE, "data", "ncu_pipes_gb300.json")
PIPE_METRICS = {"fmaheavy_active": "sm__pipe_fmaheavy_cycles_active.avg.pct_of_peak_sustained_active",
                "alu_active": "sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active",
                "issue_active": "smsp__issue_active.avg.pct_of_peak_sustained_active",
                "warps_active": "sm__warps_active.avg.pct_of_peak_sustained_active"}
# the device-code files whose change invalidates recorded per-kernel DRAM traffic
KERNEL_SOURCES = ("csrc/ks_kernels.cu", "csrc/ks_oc.cu", "csrc/ks_bconv_tc.cu", "csrc/ks_ntt_cluster.cu",
                  "csrc/ks_device.cuh", "csrc/ks_ntt_core.cuh", "csrc/ks_launch.h", "csrc/ks_oc_tower.cu",
                  "csrc/ks_cluster.cuh")


def kernel_sources_sha() -> str:
    """SHA-256 over the device-code files whose change invalidates the recorded traffic."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(HERE, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic():
    """{kernel library name: DRAM bytes per key switch} recorded on the
    current sources, else {}."""
    if not os.path.exists(TRAFFIC_PATH):
        return {}
    with open(TRAFFIC_PATH) as f:
        rec = json.load(f)
    if rec.get("sources_sha256") != kernel_sources_sha():
        return {}
    return {k: v["dram_bytes_per_ks"] for k, v in rec.get("kernels", {}).items()}


def recorded_pipes():
    """{kernel library name: {fraction name: value in [0, 1]}} recorded on
    the current sources, else {}."""
    if not os.path.exists(PIPES_PATH):
        return {}
    with open(PIPES_PATH) as f:
        rec = json.load(f)
    if rec.get("sources_sha256") != kernel_sources_sha():
        return {}
    return {k: dict(v, capture=rec.get("capture")) for k, v in rec.get("kernels", {}).items()}


def pipes_from_report(rep):
    """Per library kernel name: the pipe fractions of its first captured
    launch in an ncu report."""
    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], check=True, capture_output=True,
                         text=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    hdr = rows[0]
    ix = {h: i for i, h in enumerate(hdr)}
    per = {}
    for r in rows[2:]:
        lib = lib_name(r[ix["Kernel Name"]])
        if lib is None or lib in per:
            continue
        per[lib] = {k: round(float(r[ix[m]].replace(",", "")) / 100.0, 4) for k, m in PIPE_METRICS.items()
                    if m in ix}
    return per


def main_pipes(argv):
    """`pipes` subcommand: record pipe utilisation from an ncu report."""
    ap = argparse.ArgumentParser()
    ap.add_argument("report")
    ap.add_argument("--capture", required=True, help="the command that made the report")
    a = ap.parse_args(argv)
    rec = {"sources_sha256": kernel_sources_sha(), "capture": a.capture, "kernels": pipes_from_report(a.report)}
    with open(PIPES_PATH, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec, indent=1))


def read_launches(path):
    """[(kernel_name, grid, ns)] of the library's launches in launch order."""
    rows = []
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = r["Kernel Name"]
        m = re.search(r"\b(k_[A-Za-z0-9_]+(?:<[^()]*>)?)", name)
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
    """Per-kernel (name, launches, total ns, share) over the window [first, first+count)."""
    win = rows[first:first + count] if count else rows[first:]
    per = {}
    for name, _, ns in win:
        c, t = per.get(name, (0, 0.0))
        per[name] = (c + 1, t + ns)
    total = sum(t for _, t in per.values())
    table = sorted(((n, c, t, t / total if total else 0.0) for n, (c, t) in per.items()), key=lambda x: -x[2])
    return table, total, len(win)


def to_markdown(table, total, n):
    """The summary as a markdown table."""
    out = [f"{n} launches, {total / 1e3:.1f} us total (ncu: cold cache, serialised)", "",
           "| kernel | launches | total us | share |", "|---|---|---|---|"]
    for name, c, t, sh in table:
        out.append(f"| `{name}` | {c} | {t / 1e3:.1f} | {100 * sh:.1f}% |")
    return "\n".join(out)


# library launch names (KS_LAUNCH) of the key-switching kernels
LIB_NAMES = {"k_fwd_row": "ntt_fwd_row", "k_fwd_col": "ntt_fwd_col", "k_inv_row": "ntt_inv_row",
             "k_inv_col": "ntt_inv_col", "k_bconv_up": "bconv_up", "k_bconv_down": "bconv_down",
             "k_oc_comb_qw": "oc_comb_q", "k_oc_comb_pw": "oc_comb_p", "k_oc_comb_q": "oc_comb_q",
             "k_oc_comb_p": "oc_comb_p", "k_oc_comb_qg": "oc_comb_q", "k_oc_comb_pg": "oc_comb_p",
             "k_fwd_cl": "ntt_fwd_cl", "k_inv_cl": "ntt_inv_cl", "k_oc_rowP": "oc_row_p", "k_oc_rowQ": "oc_row_q",
             "k_apply_key": "apply_key", "k_down_final": "down_final", "k_automorph": "automorph",
             "k_bypass_copy": "bypass_copy", "k_scale": "scale", "k_oc_tower": "oc_tower",
             "k_shard_keyprod": "shard_keyprod", "k_shard_final": "shard_final"}


# kernels named by their first template argument (the stage), whatever the rest
LIB_BY_FIRST_ARG = {"k_bconv_tc": {"0": "bconv_up", "1": "bconv_down"}}


def lib_name(kernel_name):
    """Library launch name of an ncu kernel name, or None."""
    m = re.search(r"\b(k_[A-Za-z0-9_]+)(<[^()]*>)?", kernel_name)
    if not m:
        return None
    if m.group(1) in LIB_BY_FIRST_ARG and m.group(2):
        return LIB_BY_FIRST_ARG[m.group(1)].get(m.group(2)[1:-1].split(",")[0].strip())
    full = m.group(1) + (m.group(2) or "")
    return LIB_NAMES.get(full, LIB_NAMES.get(m.group(1)))


def traffic_from_report(rep, key_switches):
    """Sum dram__bytes_read.sum + dram__bytes_write.sum of every captured
    launch in an ncu report, per library kernel name, divided by the number
    of key switches the captured launches processed."""
    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], check=True, capture_output=True,
                         text=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    hdr, units = rows[0], rows[1]
    ix = {h: i for i, h in enumerate(hdr)}
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    per = {}
    for r in rows[2:]:
        lib = lib_name(r[ix["Kernel Name"]])
        if lib is None:
            continue
        b = 0.0
        for name in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            b += float(r[ix[name]].replace(",", "")) * scale[units[ix[name]]]
        c, t = per.get(lib, (0, 0.0))
        per[lib] = (c + 1, t + b)
    return {k: {"launches": c, "dram_bytes_per_ks": t / key_switches} for k, (c, t) in per.items()}


def main_traffic(argv):
    """`traffic` subcommand: record DRAM bytes per key switch from an ncu report."""
    ap = argparse.ArgumentParser()
    ap.add_argument("report")
    ap.add_argument("--key-switches", type=int, required=True)
    ap.add_argument("--capture", required=True, help="the command that made the report")
    a = ap.parse_args(argv)
    rec = {"sources_sha256": kernel_sources_sha(), "capture": a.capture, "key_switches": a.key_switches,
           "kernels": traffic_from_report(a.report, a.key_switches)}
    os.makedirs(os.path.dirname(TRAFFIC_PATH), exist_ok=True)
    with open(TRAFFIC_PATH, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec, indent=1))


def main():
    """Command line: summarise a launch list, or `traffic`."""
    import sys
    if len(sys.argv) > 1 and sys.argv[1] == "traffic":
        return main_traffic(sys.argv[2:])
    if len(sys.argv) > 1 and sys.argv[1] == "pipes":
        return main_pipes(sys.argv[2:])
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
