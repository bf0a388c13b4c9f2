"""Host-side arithmetic of bench.py: the algorithmic work per pose-atom, the roofline
fraction and the denominators (CPU only; no GPU, no oracle run)."""
import math

import bench


def test_algorithmic_counts_of_the_tucker_form():
    # energy: three two-row lerps per axis rank (9 sum r), the r1 r2 r3 contraction
    # (2 r1 r2 r3), pose transform and index (30)
    assert bench.algorithmic_flops_per_pose_atom("k_sorted_tc", (20, 20, 20)) == 16570
    assert bench.algorithmic_flops_per_pose_atom("k_sorted_tc", (18, 20, 7)) == 9 * 45 + 2 * 2520 + 30
    # energy + gradient: two core contractions, twice the lerps, the r1 r2 finishes
    g = bench.algorithmic_flops_per_pose_atom("k_sorted_tc_grad", (20, 20, 20))
    assert g == 4 * 8000 + 18 * 60 + 8 * 400 + 60
    assert bench.algorithmic_flops_per_pose_atom("k_sorted_atoms", (20, 20, 20)) is None


def test_roofline_fraction_uses_algorithmic_flops_and_device_sm_count():
    pk = {"hbm_gbs": 6786.2, "sm_max_mhz": 2070.0, "src": "measured", "sms": 152}
    timings = {"k_sorted_tc_grad": {"ms": 4.0, "launches": 2, "work": 2.0e10},
               "k_sorted_tc": {"ms": 1.0, "launches": 1, "work": 1.0e10}}
    rf = bench.roofline(timings, pk, pose_atoms_per_launch=5e6, ranks=(20, 20, 20))
    assert rf["kernel"] == "k_sorted_tc_grad" and rf["unit"] == "TFLOP/s"
    flops = (4 * 8000 + 18 * 60 + 8 * 400 + 60) * 5e6
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert math.isclose(rf["achieved"], flops / 2e-3 / 1e12, rel_tol=1e-4)
    assert math.isclose(rf["peak"], peak, rel_tol=1e-4)
    assert math.isclose(rf["frac"], rf["achieved"] / rf["peak"], rel_tol=1e-3)
    # the instruction-level model stays beside it: 1e10 ops per launch / 2 ms
    assert math.isclose(rf["instruction_model"]["achieved"], 5.0, rel_tol=1e-4)
    assert rf["avg_launch_ms"] == 2.0
    # another SM count changes the derived peak
    pk2 = dict(pk, sms=148)
    assert math.isclose(bench.fp32_pipe_peak(pk2) / bench.fp32_pipe_peak(pk), 148 / 152)


def test_traffic_is_withheld_when_the_kernel_changed(monkeypatch):
    pk = {"hbm_gbs": 6786.2, "sm_max_mhz": 2070.0, "src": "measured", "sms": 152}
    timings = {"k_sorted_tc": {"ms": 1.0, "launches": 1, "work": 1.0e10}}
    monkeypatch.setattr(bench, "TRAFFIC", {"k_sorted_tc": {"bytes_per_pose_atom": 10.0,
                                                           "sources": "not-the-current-digest",
                                                           "profile": "x.md"}})
    rf = bench.roofline(timings, pk, pose_atoms_per_launch=1e6, ranks=(20, 20, 20))
    assert rf["traffic"] is None and "changed" in rf["traffic_src"]
    monkeypatch.setattr(bench, "TRAFFIC", {"k_sorted_tc": {"bytes_per_pose_atom": 10.0,
                                                           "sources": bench.kernel_sources_digest(),
                                                           "profile": "x.md"}})
    rf = bench.roofline(timings, pk, pose_atoms_per_launch=1e6, ranks=(20, 20, 20))
    assert rf["traffic"] == 10_000_000
