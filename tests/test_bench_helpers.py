"""Host-side arithmetic of bench.py's reporting, on CPU: the walk kernel's
algorithmic HBM bytes per launch (reads: packed R, 1/R_ll, perm, the table,
z; writes: hard decisions, LLRs, PED pairs) for the bench workload, and the
fraction against a peak."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_walk_hbm_bytes_of_the_bench_workload():
    # 16x16 64-QAM, 3276 subcarriers x 14 symbols, N_pe 256, 6 bits per symbol
    n_sc, n_sym, nt, B, n_pe = 3276, 14, 16, 6, 256
    h = bench.walk_hbm(n_sc, n_sym, nt, B, n_pe, launch_ms=1.0)
    r_packed = n_sc * 136 * 8          # 16 * 17 / 2 complex64
    inv_perm = n_sc * (16 * 4 + 16)
    table = n_sc * 256 * 16
    z = n_sc * 14 * 16 * 8
    assert h["read_bytes"] == r_packed + inv_perm + table + z == 23_115_456
    hard, llr, ped2 = n_sc * 14 * 16, n_sc * 14 * 16 * 6 * 4, n_sc * 14 * 8
    assert h["write_bytes"] == hard + llr + ped2 == 18_712_512
    assert abs(h["achieved_gbs"] - (h["bytes_per_launch"] / 1e-3) / 1e9) < 1e-9
    if h["peak_gbs"]:
        assert abs(h["frac"] - h["achieved_gbs"] / h["peak_gbs"]) < 1e-12
