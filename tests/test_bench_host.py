"""Host-side pieces of bench.py (CPU): roofline constants, traffic bookkeeping, clock parsing."""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fp32_peak_is_the_unit_count_times_the_clock():
    pk = bench.peaks()
    assert abs(pk["fp32_tflops"] - 148 * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12) < 1e-9
    assert pk["hbm_gbs"] > 0


def test_flop_counts_are_the_frozen_per_pair_figures():
    m = 2 * 0.05 / 0.0375 + 1
    assert abs(bench.flops_fwd(m) - 47.33) < 0.01 and abs(bench.flops_pose(m) - 73.67) < 0.01
    mg = 8 * 0.05 / 0.0375 + 1
    assert abs(bench.flops_adj_gauss(mg) + bench.flops_pose_gauss(mg) - 242.0) < 0.01


def test_pairs_and_m_follow_the_kernel_support():
    g = {"nx": 4, "ny": 5, "nz": 6, "n_elem": 7, "n_frames": 3, "c_mm_per_us": 1.5, "fs_mhz": 40.0,
         "a0_mm": 0.05}
    pairs, m = bench.pairs_and_m(g)
    assert pairs == 4 * 5 * 6 * 7 * 3 and abs(m - (0.1 / 0.0375 + 1)) < 1e-12
    _, mg = bench.pairs_and_m(dict(g, kernel="gauss", sigma_mm=0.05))
    assert abs(mg - (0.4 / 0.0375 + 1)) < 1e-12


def test_traffic_entries_are_valid_only_for_their_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        t = json.load(fh)
    for k, e in t.items():
        if not isinstance(e, dict):
            continue
        got = bench.traffic_for(k)
        if e["src_sha"] == bench.kernel_src_hash(k):
            assert got == e["bytes_per_launch"]
        else:
            assert got is None
    assert bench.traffic_for("no_such_kernel") is None


def test_clock_summary_parses_nvidia_smi_rows(tmp_path):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clk.csv")
    with open(c.path, "w") as fh:
        fh.write("0, 2032, 2032, 550.1, 0x0, Not Active, Not Active, Not Active, Active\n")
        fh.write("0, 2010, 2032, 560.3, 0x4, Not Active, Not Active, Not Active, Not Active\n")
    s = c.summary()
    assert s["sm_max_mhz"] == 2032 and s["sm_mhz"] == pytest.approx(2021.0) and s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 2


def test_forward_shared_bytes_per_pair():
    """24 bytes per pair on the full scan (S = 4: three running-sum slots), 96 for the
    Gaussian at sigma = 0.05 mm (S = 12: its twelve weights), 56 for the Gaussian at S = 8
    (seven running-sum slots), 16 for a sphere narrower than a sample (S = 2)."""
    from paper_2604_09643_b300 import synth
    g = synth.make_geom((8, 8, 8), 0.1, 4, 1, 64)
    assert bench.fwd_smem_bytes_per_pair(g) == 24
    assert bench.fwd_smem_bytes_per_pair(dict(g, kernel="gauss", sigma_mm=0.05)) == 96
    assert bench.fwd_smem_bytes_per_pair(dict(g, kernel="gauss", sigma_mm=0.03)) == 56
    assert bench.fwd_smem_bytes_per_pair(dict(g, a0_mm=0.015)) == 16
