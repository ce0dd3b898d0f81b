"""Host-side logic checked without a GPU: the level-direction rule the
device and host loops share (compiled from the library's own header with
the host compiler), and the benchmark's algorithmic-byte count of a batched
launch (the numerator of its roofline)."""
from __future__ import annotations

import os
import subprocess
import textwrap

import pytest

import bench

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2103_13577_gb300", "csrc")

DIRECTION_PROBE = textwrap.dedent(r"""
    #define __host__
    #define __device__
    #include <cstdio>
    #include "bfs_internal.h"
    using bfs::choose_direction;
    int main() {
        const long long n = 1000000;
        // mode 0: top-down, bitmap order above n / bitmap_div frontier vertices
        printf("%d %d %d\n", choose_direction(0, false, 900, 10, 10, n, 15, 18, 0),
               choose_direction(0, false, 10, 10, 200000, n, 15, 18, 8),
               choose_direction(0, false, 10, 10, 100000, n, 15, 18, 8));
        // mode 2: bottom-up on every level
        printf("%d\n", choose_direction(2, false, 1, 1000000, 1, n, 15, 18, 0));
        // mode 1 from top-down: bottom-up once m_f * alpha > m_u
        printf("%d %d\n", choose_direction(1, false, 100, 1499, 5, n, 15, 18, 0),
               choose_direction(1, false, 100, 1500, 5, n, 15, 18, 0));
        // mode 1 from bottom-up: back to top-down once n_f * beta < n
        printf("%d %d\n", choose_direction(1, true, 1, 1, 55555, n, 15, 18, 0),
               choose_direction(1, true, 1, 1, 55556, n, 15, 18, 0));
        return 0;
    }
""")


def test_direction_rule(tmp_path):
    src = tmp_path / "probe.cpp"
    exe = tmp_path / "probe"
    src.write_text(DIRECTION_PROBE)
    try:
        subprocess.check_call(["g++", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("no host C++ compiler")
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    assert out[0].split() == ["0", "1", "0"]   # 200000 * 8 > n; 100000 * 8 < n
    assert out[1].split() == ["2"]
    assert out[2].split() == ["2", "0"]        # 100 * 15 > 1499, not > 1500
    assert out[3].split() == ["0", "2"]        # 55555 * 18 < 1e6 <= 55556 * 18


def test_batch_frontier_sums_path_graph():
    # path 0-1-2-3-4, lanes rooted at both ends: level 3 holds 3 (lane 0)
    # and 1 (lane 1), so a vertex enters the frontier once per distinct level
    import torch
    rows = torch.tensor([[0, 1, 2, 3, 4], [4, 3, 2, 1, 0], [-1, -1, -1, -1, -1]],
                        dtype=torch.int8)
    deg = torch.tensor([1, 2, 2, 2, 1], dtype=torch.int64)
    sizes, degs, reached = bench.batch_frontier_sums(rows, deg)
    assert sizes == [2, 2, 1, 2, 2]
    assert degs == [2, 4, 2, 4, 2]
    assert reached == 5
    b = bench.batch_algorithmic_bytes(sizes, degs, reached, n=5, k=3, elem=1)
    # columns 4*14 + per-entry 120*9 + sweeps 16*5*5 + init/emit 28*5 + rows 64*5 + out 3*5
    assert b == 56 + 1080 + 400 + 140 + 320 + 15


def test_batch_frontier_sums_unreached_and_isolated():
    import torch
    rows = torch.tensor([[0, -1, 1], [1, -1, 0]], dtype=torch.int32)
    deg = torch.tensor([1, 0, 1], dtype=torch.int64)
    sizes, degs, reached = bench.batch_frontier_sums(rows, deg)
    assert sizes == [2, 2] and degs == [2, 2] and reached == 2


def test_traffic_records_follow_the_kernel_sources(tmp_path):
    # the bench reports a committed ncu traffic figure only while the kernel
    # source it was captured on is unchanged
    changed = tmp_path / "kernel.cu"
    changed.write_bytes(open(bench.KERNEL_SRC, "rb").read() + b"\n// changed\n")
    assert bench.recorded_traffic(bench.TRAFFIC_FILE, str(changed)) is None
    assert bench.recorded_traffic(str(tmp_path / "missing.json")) is None
    stale = []
    for rec, src in ((bench.TRAFFIC_FILE, bench.KERNEL_SRC),
                     (bench.BATCH_TRAFFIC_FILE, bench.KERNEL_SRC),
                     (bench.PATHS_TRAFFIC_FILE, bench.PATHS_SRC)):
        value = bench.recorded_traffic(rec, src)
        if value is None:
            stale.append(os.path.basename(rec))
        else:
            assert value > 0
    if stale:
        pytest.skip("captured on an earlier kernel source (re-profile on a GPU): " + ", ".join(stale))
