"""Turns an ncu launch list (CSV from ``ncu --csv --metrics ...``) into the
short summaries kept under profiles/: per kernel its launches, total device
time and share, and -- when DRAM byte counters were captured -- the DRAM
traffic per launch of one kernel, stamped with a hash of the kernel source
so that a stale number is never reported for a changed kernel.  Also the
algorithmic bytes of a batched launch, the numerator of its roofline.

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


def batch_frontier_sums(rows, deg):
    """Frontiers of a top-down 64-root batched traversal, recovered from its
    distance rows: for every level L, |A_L| = the vertices some lane reaches
    at level L (one queue entry each, carrying its lane set) and D_L = the
    sum of their degrees (the column entries level L expands); plus R = the
    vertices any lane reaches.  rows: [k][N] distances (-1 unreached, int32
    or int8), deg: [N] out-degrees; torch tensors on one device."""
    sizes, degs = [], []
    top = int(rows.max().item())
    for level in range(top + 1):
        a = (rows == level).any(0)
        sizes.append(int(a.sum().item()))
        degs.append(int(deg[a].sum().item()))
    reached = int((rows >= 0).any(0).sum().item())
    return sizes, degs, reached


def batch_algorithmic_bytes(sizes, degs, reached: int, n: int, k: int, elem: int) -> float:
    """Bytes one top-down batched launch (bfs_batch_persistent) has to move,
    each item once:
      init      16 N                 visited/next lane-set pairs cleared
      level L   4 D_L                column entries of the frontier's rows
                + 28 |A_L|           two row offsets, queue entry (vertex + lane set)
                + 16 N               sweep reads every vertex's lane-set pair
                + 92 |A_L|           producing A_L: pair write-back, 64-byte
                                     level row, queue entry
      emit      12 N + 64 R          visited set and renumbering of every vertex,
                                     level rows of the reached ones
                + k N elem           the k distance rows
    Lane-set updates of the neighbours (atomicOr on next) and the level-row
    re-reads of vertices reached before are cache traffic, not counted."""
    per_level = sum(4 * d + 120 * a + 16 * n for a, d in zip(sizes, degs))
    return float(per_level + 16 * n + 12 * n + 64 * reached + k * n * elem)


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
