"""The TEPS definition (reading c5) pinned to the paper's Table 1: every
printed GTEPS equals edges / time within the rounding of the printed time
(times have two decimals), for the DGX-2 and both CPU columns."""
from __future__ import annotations

import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_teps.txt")


def rows():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        yield name, [float(v) for v in vals]


def test_table1_gteps_is_edges_over_time():
    n = 0
    for name, (edges_m, t_gpu, g_gpu, t_do, g_do, t_td, g_td) in rows():
        for t, g in ((t_gpu, g_gpu), (t_do, g_do), (t_td, g_td)):
            # printed time t stands for a true time in [t - 0.005, t + 0.005]
            lo, hi = edges_m / 1e3 / (t + 0.005), edges_m / 1e3 / max(t - 0.005, 1e-9)
            assert lo * 0.99 <= g <= hi * 1.01, (name, t, g, lo, hi)
        n += 1
    assert n == 9


def test_table1_speedup_columns_follow_from_times():
    # DGX2-TD / CPU-TD speedup ~ cpu_td_time / dgx2_time (GAP_kron prints 233.85)
    for name, (edges_m, t_gpu, g_gpu, t_do, g_do, t_td, g_td) in rows():
        if name == "GAP_kron":
            assert abs(g_gpu / g_td - 233.85) / 233.85 < 0.01
