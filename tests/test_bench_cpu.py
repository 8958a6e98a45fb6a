"""Host arithmetic of bench.py's JSON line: the algorithmic bytes per
cell-snapshot-stage of the tile kernel and the roofline fractions built from
them (no GPU)."""
import math

import bench


def test_algorithmic_bytes_of_the_benchmark_workload():
    # 8-block laminar pitching O-grid, FP32, 7 snapshots: (2+3+3+3)/4 x 4 vars
    # x 4 B of state, plus the 2 node coordinates per cell read once for 7 snapshots
    b = bench.algorithmic_bytes_per_unit(nv=4, s=4, dim=2, ns=7)
    assert math.isclose(b, 44.0 + 8 / 7, rel_tol=1e-15)
    # FP32 3D box, 5 snapshots: 220 B per cell-snapshot-iteration of state
    # (55 B per stage) plus 3 node coordinates per cell over 5 snapshots
    b3 = bench.algorithmic_bytes_per_unit(nv=5, s=4, dim=3, ns=5)
    assert math.isclose(b3, 55.0 + 12 / 5, rel_tol=1e-15)


def test_hbm_roofline_fraction():
    peaks = {"hbm_gbs": 6775.3}
    # one stage of 1,720,320 cell-snapshots at 51.4 B in 0.1136 ms
    r = bench.roofline(peaks, "measured", 51.4, 1720320, 0, 0.1136, "tile", None)
    assert r["units_per_launch"] == 1720320
    assert math.isclose(r["achieved"], 51.4 * 1720320 / 0.1136e-3 / 1e9, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / 6775.3, rel_tol=1e-12)
    # the persistent driver runs 4 stages per launch
    r4 = bench.roofline(peaks, "measured", 51.4, 1000, 1, 1.0, "persist", None)
    assert r4["units_per_launch"] == 4000


def test_fp32_arithmetic_peak_from_unit_counts():
    assert math.isclose(bench.FP32_PEAK_TFLOPS, 152 * 128 * 2 * 2.07e9 / 1e12, rel_tol=1e-15)
    assert 80.0 < bench.FP32_PEAK_TFLOPS < 81.0
