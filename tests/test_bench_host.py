"""Host-side logic of bench.py that needs no GPU: the roofline table (the
algorithmic bytes per unit of each stage, the dominant stage, and the DRAM
traffic scaled from the scale-workload capture)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_roofline_table_dominant_and_bytes(bench):
    n, N, G, D = 1_000_000_000, 100_000_000, 10_000_000, 250_000
    r = bench.roofline_table("scale", n, N, G, D, [5.0, 5.0], [12.0, 14.0], [10.0], "k_mrounds1", 6000.0, "measured")
    kinds = [k["kernel"] for k in r["by_kernel"]]
    assert kinds[0] == "k_compress" and kinds[2] == "k_mrounds1"
    assert r["kernel"].startswith("local aggregation")            # 13 ms mean beats 10 and 5
    assert r["algorithmic_bytes_per_launch"] == 16.0 * N + 48.0 * G + 12.0 * D
    assert r["ms_per_launch"] == 13.0
    ach = r["algorithmic_bytes_per_launch"] / 13e-3 / 1e9
    assert abs(r["achieved"] - ach) < 1e-9 * ach and abs(r["frac"] - ach / 6000.0) < 1e-12
    # traffic: 16.20 B per piece of the capture, scaled by the pieces
    assert abs(r["traffic"] - 283.246592e6 / 17479524 * N) < 1.0
    comp = r["by_kernel"][0]
    assert comp["algorithmic_bytes_per_launch"] == 8.0 * n + 12.0 * N
    # compression: 9.72 B per point of the capture, scaled by the points
    assert abs(comp["traffic"] - 1397.301728e6 / 143804766 * n) < 1.0
    assert r["by_kernel"][2]["traffic"] is None


def test_roofline_table_other_workload_has_no_traffic(bench):
    r = bench.roofline_table("multivar", 10, 5, 2, 1, [1.0], [1.0], [3.0], "k_mrounds", 100.0, "fallback")
    assert r["kernel"] == "k_mrounds" and r["traffic"] is None and r["peak_source"] == "fallback"
    assert r["algorithmic_bytes_per_launch"] == 12.125 * 2
    assert all(k["traffic"] is None for k in r["by_kernel"])
