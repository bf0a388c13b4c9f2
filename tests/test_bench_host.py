"""Host-side arithmetic of bench.py: the algorithmic work per pose-atom, the roofline
fraction and the denominators, and the multi-rank path (the slowest rank's step time on
every rank, as two gloo ranks on the CPU; the reference arm on rank 0 only).  CPU only;
no GPU, no oracle run."""
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


def _rank_main(rank, world, port, queue):
    """One CPU rank of a two-rank gloo job: its own step time in, the job's out."""
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.job_step_time(10.0 + 5.0 * rank, world, "cpu")
        dist.barrier()
        queue.put((rank, t, bench.job_throughput(1000, world, t / 1e3)))
    finally:
        dist.destroy_process_group()


def test_two_rank_job_takes_the_slowest_rank_on_every_rank():
    """The N > 1 host path of the step (world size 2, gloo on the CPU): each rank
    reports the MAX of the ranks' step times, and the job's throughput counts both
    ranks' poses over that time."""
    import multiprocessing as mp
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, t, v in got:
        assert t == 15.0
        assert math.isclose(v, 2 * 1000 / 0.015)


def test_single_rank_job_needs_no_process_group():
    assert bench.job_step_time(12.5, 1, "cpu") == 12.5
    assert math.isclose(bench.job_throughput(100000, 1, 0.0125), 8.0e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the reference arm (the oracle on the host cores) runs on rank 0;
    the other ranks return at once, before any oracle work."""
    import argparse
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(poses=100000, steps=10 ** 6, warmup=10 ** 6)
    assert bench.run_reference(args) == 0
