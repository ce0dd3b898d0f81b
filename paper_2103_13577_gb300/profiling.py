"""Turns an ncu launch list (CSV from ``ncu --csv --metrics ...``) into the
short summaries kept under profiles/: per kernel its launches, total device
time and share, and -- when DRAM byte counters were captured -- the DRAM
traffic per launch of one kernel, stamped with a hash of the kernel source
so that a stale number is never reported for a changed kernel.

Usage:
  python -m paper_2103_13577_gb300.profiling LAUNCHES.csv OUT.md \
      [--traffic-kernel REGEX --traffic-json OUT.json] [--command "..."]
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re
from collections import OrderedDict

HERE = os.path.dirname(os.path.abspath(__file__))
KERNEL_SRC = os.path.join(HERE, "csrc", "bfs_kernels.cu")


def kernel_hash() -> str:
    with open(KERNEL_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def read_launches(path: str):
    rows = list(csv.reader(open(path)))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "Metric Name" in r)
    h = rows[hdr]
    iid, iname, imet, ival, iunit = (h.index("ID"), h.index("Kernel Name"), h.index("Metric Name"),
                                     h.index("Metric Value"), h.index("Metric Unit"))
    launches = OrderedDict()
    for r in rows[hdr + 1:]:
        if len(r) < len(h):
            continue
        rec = launches.setdefault(r[iid], {"name": r[iname], "metrics": {}})
        val = float(r[ival].replace(",", ""))
        unit = r[iunit]
        scale = {"ns": 1e-9, "us": 1e-6, "usecond": 1e-6, "ms": 1e-3, "msecond": 1e-3,
                 "s": 1.0, "second": 1.0, "nsecond": 1e-9, "byte": 1.0, "Kbyte": 1e3,
                 "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}.get(unit, 1.0)
        rec["metrics"][r[imet]] = val * scale
    return launches


def short_name(name: str) -> str:
    return re.sub(r"\(.*", "", name).replace("void ", "").strip()


def summarize(path: str, out_md: str, traffic_kernel: str | None, traffic_json: str | None,
              command: str) -> None:
    launches = read_launches(path)
    per = OrderedDict()
    for rec in launches.values():
        k = short_name(rec["name"])
        p = per.setdefault(k, {"launches": 0, "time_s": 0.0, "dram": []})
        p["launches"] += 1
        p["time_s"] += rec["metrics"].get("gpu__time_duration.sum", 0.0)
        if "dram__bytes_read.sum" in rec["metrics"]:
            p["dram"].append(rec["metrics"]["dram__bytes_read.sum"] +
                             rec["metrics"].get("dram__bytes_write.sum", 0.0))
    total = sum(p["time_s"] for p in per.values()) or 1.0
    lines = ["# ncu launch list summary", "", f"Command: `{command}`", "",
             "Per-launch times are cold-cache and serialised under ncu; compare shares.", "",
             "| kernel | launches | total time (ms) | share | DRAM bytes / launch |",
             "|---|---|---|---|---|"]
    for k, p in sorted(per.items(), key=lambda kv: -kv[1]["time_s"]):
        dram = "%.3e" % (sum(p["dram"]) / len(p["dram"])) if p["dram"] else "-"
        lines.append(f"| {k} | {p['launches']} | {p['time_s'] * 1e3:.3f} | "
                     f"{p['time_s'] / total * 100:.1f}% | {dram} |")
    with open(out_md, "w") as f:
        f.write("\n".join(lines) + "\n")
    if traffic_kernel and traffic_json:
        rx = re.compile(traffic_kernel)
        vals = [p["dram"] for k, p in per.items() if rx.search(k) and p["dram"]]
        flat = [x for v in vals for x in v]
        if flat:
            with open(traffic_json, "w") as f:
                json.dump({"kernel": traffic_kernel, "launches": len(flat),
                           "dram_bytes_per_launch": sum(flat) / len(flat),
                           "kernel_sha256_16": kernel_hash(), "command": command}, f, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("out_md")
    ap.add_argument("--traffic-kernel")
    ap.add_argument("--traffic-json")
    ap.add_argument("--command", default="")
    a = ap.parse_args()
    summarize(a.csv, a.out_md, a.traffic_kernel, a.traffic_json, a.command)


if __name__ == "__main__":
    main()
