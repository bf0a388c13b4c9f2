#!/usr/bin/env python
"""Throughput of the RS-tensor pose-energy path on GB300.

One step = the whole hot path over one batch of the protein-scale workload:
Algorithm TEP (sinc table, cell list, long-range factors, RHOSVD to Tucker rank
<= 20) for N=3000 protein atoms on an n=1025 grid, then Algorithm PLIE energies,
vdW flags and exact rigid-body gradients for P=1e5 poses of a 50-atom ligand.
value = poses per second through that step (whole job over all ranks).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "poses/sec at <=1e-5 rel err vs FP64 oracle; served p50/p99 latency vs plain"
UNIT = "poses/s"
WORKLOAD = ("plain_protein: N=3000 charges on a jittered 1.5 A lattice in a (20,14,10) A "
            "ellipsoid, 8% +-1; ligand L=50; n=1025 on [-64,64]^3; R_l=20; Tucker rank <= 20; "
            "P=1e5 poses, |t| in [10,30] A; step = TEP build + energies + gradients")
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--poses", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="step mode: skip the served, batched and PGD sub-measurements")
    ap.add_argument("--mode", choices=["step", "build", "batch", "pgd", "serve", "fd", "ppiem", "localbox", "complex"],
                    default="step",
                    help="step: the protein-scale hot-path step (default); batch: 64 uneven "
                         "pairs in one persistent graph launch vs 64 plain launches; pgd: "
                         "projected gradient descent; serve: Poisson request stream through "
                         "the serving loop vs the plain per-request path; fd: the paper's "
                         "finite-difference forces and rigid-cluster resultants vs the exact "
                         "gradient on the same poses; ppiem: the pose scan of Algorithm PPIEM "
                         "(contact search, energies, minima); localbox: energies through a "
                         "local-box handle (scheme C) vs the global handle; complex: a two-molecule "
                         "complex (Eq. EnergySum_Mcomplex) vs the union molecule, and Galerkin vs "
                         "collocation factors on the small canonical workload")
    ap.add_argument("--scan", type=str, default="16,32,12",
                    help="ppiem: n_theta,n_phi,m_L (directions n_theta x n_phi; m_L^3/2 rotations)")
    ap.add_argument("--pairs", type=int, default=64)
    ap.add_argument("--pair-poses", type=int, default=10_000, help="batch: poses per pair")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: requests per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--serve-n-max", type=int, default=16385, help="serve: largest grid")
    ap.add_argument("--group-min-atoms", type=int, default=None,
                    help="serve: pose-atoms from which a request joins the cell-grouped pipeline")
    ap.add_argument("--group-atoms-per-cell", type=float, default=None,
                    help="serve: pose-atoms per axis-3 cell from which a request is grouped")
    return ap.parse_args()


def quat_to_rotvec(q: np.ndarray) -> np.ndarray:
    """Rotation vector of a unit quaternion (w, x, y, z): input preparation for the
    gradient pass, the same rotations as the energy pass."""
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    q = np.where(q[:, :1] < 0, -q, q)
    v = q[:, 1:]
    s = np.linalg.norm(v, axis=1)
    ang = 2.0 * np.arctan2(s, q[:, 0])
    scale = np.where(s > 1e-12, ang / np.where(s > 1e-12, s, 1.0), 2.0)
    return v * scale[:, None]


def workload(P: int, seed: int = 1):
    import workloads as W
    w = W.plain_protein(seed=seed, P=P)
    return w, quat_to_rotvec(w.quat)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={SMI_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[4:]))
                except ValueError:
                    continue
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[2][1:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ roofline
def peaks(sm_count: int | None = None) -> dict:
    """Denominators: HBM copy bandwidth from MEASURED_PEAKS.json (measured), and the
    FP32 pipe derived from the SM count, 128 FP32 lanes per SM and the maximum SM
    clock (no FP32 figure is measured)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sms = sm_count if sm_count else 152
    try:
        m = json.load(open(path))
        return {"hbm_gbs": m["hbm_gbs"], "sm_max_mhz": m.get("sm_max_mhz", 2070.0), "src": "measured",
                "sms": sms}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "src": "fallback", "sms": sms}


def fp32_pipe_peak(pk: dict) -> float:
    """FP32 pipe instructions per second (FADD/FMUL/FFMA = 1 each), in T op/s."""
    return pk["sms"] * 128 * pk["sm_max_mhz"] * 1e6 / 1e12


# Kernel -> (bound, unit of its reported work).  "fp32ops": FP32 pipe operations
# (FADD, FMUL, FFMA each 1), peak SMs x 128 lanes x max SM clock; "fp32": FP32
# flops (FMA = 2), peak twice that; FP64 ALU peak: 1.25 TFLOP/s (GB300 table).
KERNEL_KIND = {
    "k_eval_wform": ("alu", "fp32ops"), "k_eval_wform_grad": ("alu", "fp32ops"),
    "k_eval_canon": ("alu", "fp32"), "k_eval_canon_grad": ("alu", "fp32"),
    "k_sorted_wform": ("alu", "fp32ops"), "k_sorted_wform_grad": ("alu", "fp32ops"),
    "k_sorted_tc": ("alu", "fp32ops"), "k_sorted_tc_grad": ("alu", "fp32ops"), "k_group_tc": ("alu", "fp32ops"),
    "k_sorted_atoms": ("alu", "fp32ops"), "k_sorted_atoms_grad": ("alu", "fp32ops"),
    "k_project": ("alu", "fp32ops"), "k_core": ("alu", "fp32ops"), "k_gauss_dsum": ("alu", "fp32ops"),
    "k_gram": ("alu", "fp32ops"), "k_gemm_gq": ("alu", "fp32ops"), "k_canon_factors": ("hbm", "bytes"),
}

# Pose kernels whose unit is one pose-atom (one ligand atom of one pose).
POSE_ATOM_KERNELS = ("k_sorted_tc", "k_sorted_tc_grad", "k_sorted_wform", "k_sorted_wform_grad",
                     "k_sorted_atoms", "k_sorted_atoms_grad")

# DRAM bytes (read + write) per pose-atom from one ncu capture of the kernel at the
# bench's own size (one-pass DRAM metrics, so the full-size launch is captured), with
# the digest of the kernel's sources at that capture; a kernel whose sources changed
# since reports traffic null.
TRAFFIC = {
    name: {"bytes_per_pose_atom": b, "sources": "5cf7801ef109403d",
           "profile": "profiles/pose_kernels_dram_protein_p100000.md"}
    for name, b in (("k_sorted_tc_grad", 223.3), ("k_sorted_tc", 112.0), ("k_sorted_atoms_grad", 90.8),
                    ("k_sorted_atoms", 71.4))
}
TRAFFIC_SOURCES = ("rs_sorted.cu", "rs_sorted_dev.cuh", "rs_tc.cuh", "rs_tc_dev.cuh", "rs_pose_dev.cuh",
                   "rs_common.cuh")


def kernel_sources_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2510_26611_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def algorithmic_flops_per_pose_atom(name: str, ranks) -> float | None:
    """FP32 flops one pose-atom needs by the Tucker form's own arithmetic (FMA = 2):
    energy 9 (r1 + r2 + r3) + 2 r1 r2 r3 + 30 (three two-row lerps, the r1 r2 r3 core
    contraction, pose transform and index); energy and gradient together
    4 r1 r2 r3 + 18 (r1 + r2 + r3) + 8 r1 r2 + 60 (the core contracted with the lerped
    axis-3 row and with its slope, both lerps of every axis, the r1 r2 finish of the
    value and the three partials, transform, torque and chain rule)."""
    r1, r2, r3 = ranks
    if name in ("k_sorted_tc", "k_sorted_wform"):
        return 9.0 * (r1 + r2 + r3) + 2.0 * r1 * r2 * r3 + 30.0
    if name in ("k_sorted_tc_grad", "k_sorted_wform_grad"):
        return 4.0 * r1 * r2 * r3 + 18.0 * (r1 + r2 + r3) + 8.0 * r1 * r2 + 60.0
    return None


def roofline(timings: dict, pk: dict, name: str | None = None, pose_atoms_per_launch: float | None = None,
             ranks=None) -> dict:
    """Roofline of the kernel with the largest timed share (or of `name`).

    achieved = the kernel's algorithmic FP32 flops per launch (pose-atoms per launch x
    the per-pose-atom count of the Tucker form) / its average launch time, against the
    FP32 FMA peak; the library's instruction-level work model is reported beside it."""
    if not timings or (name is not None and name not in timings):
        return None
    if name is None:
        name, rec = max(timings.items(), key=lambda kv: kv[1]["ms"])
    else:
        rec = timings[name]
    bound, unit = KERNEL_KIND.get(name, ("alu", "fp32"))
    per_launch_s = rec["ms"] / 1e3 / max(rec["launches"], 1)
    work = rec["work"] / max(rec["launches"], 1)
    if unit == "bytes":
        ach, peak, u = work / per_launch_s / 1e9, pk["hbm_gbs"], "GB/s"
        note = "HBM, measured copy bandwidth"
    elif unit == "fp64":
        ach, peak, u = work / per_launch_s / 1e12, 1.25, "TFLOP/s"
        note = "FP64 ALU, nominal 1.25 TFLOP/s"
    elif unit == "fp32ops":
        ach = work / per_launch_s / 1e12
        peak = fp32_pipe_peak(pk)
        u = "Top/s"
        note = f"FP32 pipe, {pk['sms']} SMs x 128 lanes x max SM clock (FADD/FMUL/FFMA = 1 op)"
    else:
        ach = work / per_launch_s / 1e12
        peak = 2 * fp32_pipe_peak(pk)
        u = "TFLOP/s"
        note = f"FP32 ALU, {pk['sms']} SMs x 128 lanes x 2 x max SM clock"
    total = sum(r["ms"] for r in timings.values())
    instr = {"achieved": round(ach, 4), "peak": round(peak, 3), "unit": u, "frac": round(ach / peak, 4),
             "peak_src": note + f" ({pk['src']} clock)", "work": "the library's instruction-level work model"}
    out = {"kernel": name, "bound": bound, "achieved": instr["achieved"], "peak": instr["peak"], "unit": u,
           "frac": instr["frac"], "traffic": None, "peak_src": instr["peak_src"],
           "avg_launch_ms": round(per_launch_s * 1e3, 4),
           "share_of_timed_kernels": round(rec["ms"] / total, 4) if total > 0 else None}
    alg = algorithmic_flops_per_pose_atom(name, ranks) if ranks else None
    if alg is not None and pose_atoms_per_launch:
        flops = alg * pose_atoms_per_launch
        a = flops / per_launch_s / 1e12
        p = 2 * fp32_pipe_peak(pk)
        out.update({"bound": "alu", "achieved": round(a, 4), "peak": round(p, 3), "unit": "TFLOP/s",
                    "frac": round(a / p, 4),
                    "peak_src": (f"FP32 FMA, {pk['sms']} SMs x 128 lanes x 2 flops x max SM clock "
                                 f"(derived from unit counts and the {pk['src']} clock)"),
                    "work": (f"algorithmic: {alg:.0f} FP32 flops per pose-atom (Tucker ranks "
                             f"{tuple(ranks)}) x {pose_atoms_per_launch:.0f} pose-atoms per launch"),
                    "instruction_model": instr})
        t = TRAFFIC.get(name)
        if t is not None:
            if t["sources"] == kernel_sources_digest():
                out["traffic"] = round(t["bytes_per_pose_atom"] * pose_atoms_per_launch)
                out["traffic_src"] = t["profile"]
            else:
                out["traffic_src"] = "kernel changed since its ncu capture: traffic withheld"
    return out


# ------------------------------------------------------------------ CPU baseline (the oracle)
# Runs in its own process on the host cores only (CUDA hidden).  One step of the same
# kind as the GPU step on a bounded sample: one FP64 TEP build of the protein, then
# energies and gradients of the first P_s poses.  Optionally it also reports, on the
# first P_e poses, the errors of the method against exact Coulomb, of the Tucker
# rank cap against the unreduced RS potential, and of the GPU's energies (read from a
# file) against the oracle's reduced form.
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle as O
from bench import workload
P_full, P_s, P_e, gpu_path = {P}, {Ps}, {Pe}, {gpu!r}
w, rv = workload(P_full)
idx = np.arange(P_s)
t0 = time.perf_counter()
m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=w.tucker_cap,
                  keep_canonical=P_e > 0)
t1 = time.perf_counter()
O.pose_energies(m, w.lig_xyz, w.lig_q, w.quat[idx], w.trans[idx])
t2 = time.perf_counter()
O.pose_gradients(m, w.lig_xyz, w.lig_q, rv[idx], w.trans[idx])
t3 = time.perf_counter()
out = {{"build_s": t1 - t0, "energy_s": t2 - t1, "grad_s": t3 - t2}}
if P_e > 0:
    sl = slice(0, P_e)
    q, t = w.quat[sl], w.trans[sl]
    tuck = O.pose_energies(m, w.lig_xyz, w.lig_q, q, t)
    m.kind = "canonical"
    full = O.pose_energies(m, w.lig_xyz, w.lig_q, q, t)
    coul = O.coulomb_energies(w.prot_xyz, w.prot_q, w.lig_xyz, w.lig_q, q, t)
    scale = O.tolerance_scale(full["E"], full["S_ref"])
    feas = full["flags"] == 0
    def stats(a, b):
        e = np.abs(a - b) / scale
        r = {{"median": float(np.median(e)), "max": float(e.max())}}
        if feas.any():
            r.update({{"feasible_median": float(np.median(e[feas])), "feasible_max": float(e[feas].max())}})
        return r
    err = {{"poses": P_e, "feasible": int(feas.sum()),
            "denominator": "max(|E_RS|, 1e-2 sum_j |q_j phi_RS(x_j)|) of the unreduced RS energy",
            "rs_unreduced_vs_coulomb": stats(full["E"], coul),
            "tucker_vs_rs_unreduced": stats(tuck["E"], full["E"]),
            "tucker_vs_coulomb": stats(tuck["E"], coul)}}
    if gpu_path:
        g = np.load(gpu_path)[:P_e]
        ts = O.tolerance_scale(tuck["E"], tuck["S_ref"])
        eg = np.abs(g - tuck["E"]) / ts
        err["gpu_vs_oracle_tucker"] = {{"median": float(np.median(eg)), "max": float(eg.max()),
                                        "denominator": "max(|E|, 1e-2 S) of the oracle's Tucker form"}}
        err["gpu_vs_coulomb"] = stats(g, coul)
    out["errors"] = err
print(json.dumps(out))
"""


def oracle_sample(P: int, P_s: int, threads: int, P_e: int = 0, gpu_path: str = "") -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = ORACLE_SNIPPET.format(root=ROOT, P=P, Ps=P_s, Pe=P_e, gpu=gpu_path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    t = json.loads(r.stdout.strip().splitlines()[-1])
    step_s = t["build_s"] + t["energy_s"] + t["grad_s"]
    per_pose = (t["energy_s"] + t["grad_s"]) / P_s
    return {"value": P_s / step_s, "step_s": step_s, "timings": t, "P_s": P_s,
            "full_workload_estimate": P / (t["build_s"] + per_pose * P)}


CPU_SAMPLE_POSES = 10_000     # the CPU-baseline step: one build + this many poses
REF_SAMPLE_POSES = 4_000      # the reference arm's step (K + W of them must end in minutes)
ERROR_SAMPLE_POSES = 100      # poses for the error report (unreduced RS form: rank 60000)


def cpu_baseline(P: int, gpu_path: str = "") -> tuple[dict, dict | None]:
    cores = os.cpu_count() or 1
    r = oracle_sample(P, CPU_SAMPLE_POSES, cores, P_e=ERROR_SAMPLE_POSES, gpu_path=gpu_path)
    t = r["timings"]
    cpu = {"value": round(r["value"], 3), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": (f"one step of the same kind as the GPU step, measured: one FP64 TEP build "
                      f"(RHOSVD) plus energies and gradients of the first {CPU_SAMPLE_POSES} of the "
                      f"{P} poses; value = {CPU_SAMPLE_POSES} poses / measured step time; "
                      f"numpy/BLAS threads={cores}"),
           "ms_per_step": round(1e3 * r["step_s"], 1),
           "timings_s": {k: round(v, 3) for k, v in t.items() if k.endswith("_s")},
           "full_workload_estimate": {
               "value": round(r["full_workload_estimate"], 3),
               "how": f"one build + per-pose time x {P} poses (estimate, not measured)"}}
    return cpu, t.get("errors")
# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle as it stands on the host cores, on this arm's workload, metric and
    unit: each step is one FP64 TEP build plus energies and gradients of the first
    REF_SAMPLE_POSES poses (a bounded sample of the 1e5-pose step), timed as a whole;
    value = poses evaluated / measured time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    P = args.poses
    cores = os.cpu_count() or 1
    P_s = min(REF_SAMPLE_POSES, P)
    steps_s, est = [], []
    t_all = time.perf_counter()
    for it in range(args.warmup + args.steps):
        r = oracle_sample(P, P_s, cores)
        if it >= args.warmup:
            steps_s.append(r["step_s"])
            est.append(r["full_workload_estimate"])
    wall = time.perf_counter() - t_all
    value = P_s * len(steps_s) / sum(steps_s)
    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * statistics.mean(steps_s), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "poses": P, "poses_evaluated_per_step": P_s},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores,
                             "kind": "oracle",
                             "sample": (f"each step, measured: one FP64 TEP build plus energies and "
                                        f"gradients of the first {P_s} of the {P} poses; value = "
                                        f"{P_s} x steps / measured time; numpy/BLAS threads={cores}")},
            "full_workload_estimate": {
                "value": round(statistics.mean(est), 3),
                "how": f"one build + per-pose time x {P} poses (estimate, not measured)"},
            "wall_s": round(wall, 1),
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ batching mode
def measure_batch(args) -> dict:
    """64 protein-ligand pairs (N log-uniform in [500, 20000], L in [10, 200], n matched
    to the box), 1e4 poses each: one persistent graph-captured launch against 64
    sequential plain launches."""
    import torch
    import workloads as W
    from paper_2510_26611_gb300 import lib
    dev = torch.device("cuda", 0)
    ctx = lib.Context(0)
    ws = W.batch_pairs(seed=2, pairs=args.pairs, P=args.pair_poses)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    t0 = time.perf_counter()
    prots, pairs = [], []
    for w in ws:
        prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
        prots.append(lib.rs_build_protein(ctx.handle, T(w.prot_xyz), T(w.prot_q), prm))
        pairs.append(dict(prot=prots[-1], lig_xyz=T(w.lig_xyz), lig_q=T(w.lig_q), quat=T(w.quat),
                          trans=T(w.trans), E_out=torch.empty(w.P, dtype=torch.float64, device=dev),
                          flags_out=torch.empty(w.P, dtype=torch.uint8, device=dev)))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    b, keep = lib.rs_batch_create(ctx.handle, pairs, autotune=True)
    info = lib.rs_batch_get_info(b)
    E2 = [torch.empty_like(p["E_out"]) for p in pairs]
    F2 = [torch.empty_like(p["flags_out"]) for p in pairs]

    def plain():
        for p, e, f in zip(pairs, E2, F2):
            lib.rs_energy_poses(ctx.handle, p["prot"], p["lig_xyz"], p["lig_q"], p["quat"],
                                p["trans"], E_out=e, flags_out=f)

    def batched():
        lib.rs_batch_run(b)

    def timeit(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for a, c in ev:
            a.record()
            fn()
            c.record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(c) for a, c in ev) / args.steps

    with ClockSampler(0) as clk:
        ms_plain = timeit(plain)
        ms_batch = timeit(batched)
    clocks = clk.summary()
    # batched vs plain: flags identical; energies equal, or within the W-form path
    # tolerance where the two take different long-range kernels (relative to
    # max(|E|, median |E|) per pair)
    same_flags = all(torch.equal(p["flags_out"], f) for p, f in zip(pairs, F2))
    bitwise = all(torch.equal(p["E_out"], e) for p, e in zip(pairs, E2))
    rel = 0.0
    for p, e in zip(pairs, E2):
        if e.numel():
            ref = e.abs()
            scale = torch.clamp(ref, min=float(ref.median()))
            rel = max(rel, float(((p["E_out"] - e).abs() / scale).max()))
    P_tot = sum(w.P for w in ws)
    atoms = sum(w.P * w.L for w in ws)
    line = {"metric": "batched poses/s, 64 uneven pairs in one persistent graph launch",
            "value": round(P_tot / (ms_batch / 1e3), 3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_batch, 4),
            "higher_is_better": True, "data": "synthetic",
            "plain": {"value": round(P_tot / (ms_plain / 1e3), 3), "ms_per_step": round(ms_plain, 4),
                      "launches": len(pairs)},
            "speedup_vs_plain": round(ms_plain / ms_batch, 3), "flags_equal_to_plain": bool(same_flags),
            "energies_bitwise_equal_to_plain": bool(bitwise), "max_rel_diff_to_plain": rel,
            "config": {"workload": "batch_pairs: N log-uniform [500,20000], L uniform [10,200], "
                                   "n in {513,1025,2049,4097} by box quartile, "
                                   f"{args.pair_poses} poses per pair, Tucker rank <= 20",
                       "pairs": len(ws), "poses": P_tot, "atom_evaluations": atoms,
                       "n_hist": {str(n): sum(1 for w in ws if w.n == n) for n in sorted({w.n for w in ws})}},
            "batch_info": info, "build_s_total": round(build_s, 3),
            "launch_calls": {"batched": 1, "plain": len(pairs)}, "clocks": clocks}
    lib.rs_batch_free(b)
    for h in prots:
        lib.rs_protein_free(h)
    ctx.close()
    return line


def run_batch(args):
    print(json.dumps(measure_batch(args)), flush=True)
    return 0


# ------------------------------------------------------------------ build mode
def run_build(args):
    """Algorithm TEP alone: the protein-scale Tucker build (N=3000, n=1025, rank <= 20),
    timed per build with CUDA events, then once more per kernel (timing events on)."""
    import torch
    from paper_2510_26611_gb300 import lib
    dev = torch.device("cuda", 0)
    w, _ = workload(16)
    ctx = lib.Context(0)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    xyz, q = T(w.prot_xyz), T(w.prot_q)
    prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
    for _ in range(args.warmup):
        lib.rs_protein_free(lib.rs_build_protein(ctx.handle, xyz, q, prm))
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(0) as clk:
        for a, b in ev:
            a.record()
            lib.rs_protein_free(lib.rs_build_protein(ctx.handle, xyz, q, prm))
            b.record()
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    lib.rs_timing_reset()
    lib.rs_timing_enable(2)
    h = lib.rs_build_protein(ctx.handle, xyz, q, prm)
    info = lib.rs_protein_get_info(h)
    lib.rs_protein_free(h)
    torch.cuda.synchronize()
    kernels = {k: {"ms": round(v["ms"], 4), "launches": v["launches"]}
               for k, v in sorted(lib.rs_timing_all().items(), key=lambda kv: -kv[1]["ms"])}
    lib.rs_timing_enable(0)
    line = {"metric": "Tucker build (Algorithm TEP) time", "value": round(ms, 4), "unit": "ms",
            "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": WORKLOAD.split("; P=")[0], "n": w.n, "protein_atoms": w.N},
            "ranks": info["rank"], "clocks": clk.summary(),
            "kernels_one_build_with_timing_events": kernels}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# ------------------------------------------------------------------ differentiation mode
def measure_pgd(args) -> dict:
    """Constrained minimisation (Eq. Energy_Min): protein N=10000, ligand L=100, n=2049,
    4096 feasible starting poses, 50 projected-gradient steps (adjoint + backtracking)."""
    import torch
    import workloads as W
    from paper_2510_26611_gb300 import lib
    dev = torch.device("cuda", 0)
    ctx = lib.Context(0)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    holder = {}

    def feasible(qq, tt):
        w0 = holder["w"]
        E, f = lib.rs_energy_poses(ctx.handle, holder["prot"], T(w0.lig_xyz), T(w0.lig_q), T(qq), T(tt))
        return f.cpu().numpy() == 0

    # protein and ligand first (no poses), then rejection-sample feasible poses
    w = W.pgd_start(P=1)
    holder["w"] = w
    prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
    t0 = time.perf_counter()
    holder["prot"] = lib.rs_build_protein(ctx.handle, T(w.prot_xyz), T(w.prot_q), prm)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    w = W.pgd_start(P=4096, feasible=feasible)
    rv0 = W.random_rotvecs(np.random.default_rng(7), w.P)
    # the rotations of the sampled quaternions, as rotation vectors
    rv0 = quat_to_rotvec(w.quat)
    lx, lq = T(w.lig_xyz), T(w.lig_q)
    nsteps = 50
    rv, tr = T(rv0), T(w.trans)
    lib.rs_pgd_run(ctx.handle, holder["prot"], lx, lq, rv.clone(), tr.clone(), 2)  # warm-up
    E0, f0 = lib.rs_energy_poses(ctx.handle, holder["prot"], lx, lq, T(w.quat), T(w.trans))
    torch.cuda.synchronize()
    launches0 = lib.rs_stats_kernel_launches()
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        a.record()
        E, f, acc = lib.rs_pgd_run(ctx.handle, holder["prot"], lx, lq, rv, tr, nsteps)
        c.record()
        torch.cuda.synchronize()
    clocks = clk.summary()
    ms = a.elapsed_time(c)
    launches = lib.rs_stats_kernel_launches() - launches0
    # what one step is made of: a gradient pass and an energy pass over all poses
    # (per-kernel device times, timing events on; not part of the timed run)
    lib.rs_timing_reset()
    lib.rs_timing_enable(2)
    for _ in range(5):
        lib.rs_energy_grad_poses(ctx.handle, holder["prot"], lx, lq, rv, tr)
        lib.rs_energy_poses(ctx.handle, holder["prot"], lx, lq, T(w.quat), tr)
    torch.cuda.synchronize()
    kernels = {k: round(v["ms"] / 5, 4) for k, v in
               sorted(lib.rs_timing_all().items(), key=lambda kv: -kv[1]["ms"])}
    lib.rs_timing_enable(0)
    E0, E1 = E0.cpu().numpy(), E.cpu().numpy()
    line = {"metric": "gradients/s through projected gradient descent (Eq. Energy_Min)",
            "value": round(w.P * nsteps / (ms / 1e3), 3), "unit": "pose-gradients/s", "n_gpus": 1,
            "steps": nsteps, "ms_total": round(ms, 3), "ms_per_pgd_step": round(ms / nsteps, 4),
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "pgd_start: N=10000 on a jittered lattice sphere, L=100, n=2049, "
                                   "b = r_p + 2 r_l + 8, Tucker rank <= 20, 4096 feasible starting "
                                   "poses (rejection sampling on the GPU flags), 50 steps, "
                                   "eta_t = 0.1 A, eta_r = 0.02 rad, <= 5 halvings",
                       "poses": w.P},
            "result": {"mean_E_start": float(E0.mean()), "mean_E_end": float(E1.mean()),
                       "all_final_feasible": bool((f.cpu().numpy() == 0).all()),
                       "accepted_last_step": float((acc.cpu().numpy() >= 0).mean())},
            "gpu_launches": int(launches), "build_s": round(build_s, 3),
            "kernels_ms_one_gradient_and_one_energy_pass": kernels, "clocks": clocks}
    lib.rs_protein_free(holder["prot"])
    ctx.close()
    return line


def run_pgd(args):
    print(json.dumps(measure_pgd(args)), flush=True)
    return 0


def _left_jacobian(w: np.ndarray) -> np.ndarray:
    """SO(3) left Jacobian of rotation vectors (Sola et al. 2018), for comparing the
    moment of the finite-difference forces with dE/dw; host-side analysis only."""
    th = np.linalg.norm(w, axis=1)
    K = np.zeros((w.shape[0], 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -w[:, 2], w[:, 1], -w[:, 0]
    K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = w[:, 2], -w[:, 1], w[:, 0]
    small = th < 1e-4
    ts = np.where(small, 1.0, th)
    B = np.where(small, 0.5 - th ** 2 / 24, (1 - np.cos(ts)) / ts ** 2)
    C = np.where(small, 1.0 / 6 - th ** 2 / 120, (ts - np.sin(ts)) / ts ** 3)
    return np.eye(3)[None] + B[:, None, None] * K + C[:, None, None] * (K @ K)


def run_fd(args):
    """The paper's finite-difference force (Eq. differ_ligand, four potential
    evaluations per atom) with its radial/tangential resultants (Eq. Field_Xcenter,
    Eq. Field_phi), timed beside the exact adjoint gradient on the same poses of the
    protein-scale workload, and the relative deviation of each from the adjoint."""
    import torch
    from paper_2510_26611_gb300 import lib
    dev = torch.device("cuda", 0)
    P = args.poses
    w, rv = workload(P, seed=1)
    ctx = lib.Context(0)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
    prot = lib.Protein(ctx, T(w.prot_xyz), T(w.prot_q), prm)
    lx, lq, rvec, trans = T(w.lig_xyz), T(w.lig_q), T(rv), T(w.trans)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        l0 = lib.rs_stats_kernel_launches()
        with ClockSampler(0) as clk:
            for i in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                ev[i][0].record()
                out = fn()
                ev[i][1].record()
            torch.cuda.synchronize()
        launches = (lib.rs_stats_kernel_launches() - l0) // args.steps
        return sum(a.elapsed_time(b) for a, b in ev) / args.steps, out, clk.summary(), launches

    ms_fd, fd, clocks, launches_fd = timed(lambda: prot.fd_forces(lx, lq, rvec, trans))
    ms_ex, ex, _, launches_ex = timed(lambda: prot.energies_grad(lx, lq, rvec, trans))
    lib.rs_timing_reset()
    lib.rs_timing_enable(2)
    for _ in range(3):
        prot.fd_forces(lx, lq, rvec, trans)
    torch.cuda.synchronize()
    kernels = {k: round(v["ms"] / 3, 4) for k, v in
               sorted(lib.rs_timing_all().items(), key=lambda kv: -kv[1]["ms"])}
    lib.rs_timing_enable(0)
    fd = {k: v.cpu().numpy() for k, v in fd.items()}
    E, gt, gw, f = (x.cpu().numpy() for x in ex)
    ok = f == 0
    nt = np.linalg.norm(gt, axis=1)
    nw = np.linalg.norm(gw, axis=1)
    rel = lambda a, b, n: np.linalg.norm(a - b, axis=1)[ok] / n[ok]
    dw_fd = np.einsum("pji,pj->pi", _left_jacobian(rv), fd["M"])
    yc = w.lig_xyz - w.lig_xyz.mean(axis=0)
    r0 = float(np.sqrt((yc * yc).sum(axis=1).mean()))
    stats = lambda e: {"median": float(np.median(e)), "p95": float(np.percentile(e, 95)), "max": float(e.max())}
    line = {"metric": "finite-difference pose forces/s (Eq. differ_ligand + rigid-cluster resultants)",
            "value": round(P / (ms_fd / 1e3), 3), "unit": "pose-forces/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_fd, 4),
            "higher_is_better": True, "data": "synthetic",
            "dtype": "f64 build, f32-pair + bf16-slice tensor-core evaluation",
            "config": {"workload": "plain_protein: N=3000 (1.5 A lattice in a (20,14,10) A ellipsoid), "
                                   "L=50, n=1025 on [-64,64]^3, Tucker rank <= 20, P poses (uniform "
                                   "rotations as rotation vectors), |t| in [10,30] A; h = grid step, "
                                   "r0 = RMS ligand radius",
                       "poses": P, "l2": "flushed between steps (256 MiB write, outside the timed events)"},
            "exact_adjoint": {"value": round(P / (ms_ex / 1e3), 3), "unit": "pose-gradients/s",
                              "ms_per_step": round(ms_ex, 4), "gpu_launches": int(launches_ex)},
            "fd_over_exact_time": round(ms_fd / ms_ex, 3),
            "deviation_from_exact_adjoint_feasible_poses": {
                "poses": int(ok.sum()),
                "E_max_rel": float((np.abs(fd["E"] - E)[ok] / np.maximum(np.abs(E[ok]), 1e-300)).max()),
                "Fsum_vs_dE_dt": stats(rel(fd["F"], gt, nt)),
                "F0_radial_only_vs_dE_dt": stats(rel(fd["F0"], gt, nt)),
                "JT_M_vs_dE_dw": stats(rel(dw_fd, gw, nw)),
                # the tangential resultant read as a plain vector sum (Eq. Field_phi) against
                # the moment it stands for: r0 |Fphi| / |M| (1 only when the moved
                # tangential parts are parallel)
                "r0_Fphi_over_moment": stats(r0 * np.linalg.norm(fd["Fphi"], axis=1)[ok] /
                                             np.maximum(np.linalg.norm(fd["M"], axis=1)[ok], 1e-300)),
            },
            "gpu_launches": int(launches_fd), "clocks": clocks, "kernels_ms_per_call": kernels}
    print(json.dumps(line), flush=True)
    prot.close()
    ctx.close()
    return 0


def run_ppiem(args):
    """Pose scan of Algorithm PPIEM on the protein-scale workload: every orbit
    direction x self-rotation is brought to first contact along its approach line
    (A3), its energy evaluated (A4, A5), and the best rotation and local minima per
    direction found (A6).  Device buffers; the timed region is one whole scan."""
    import torch
    import workloads as W
    from paper_2510_26611_gb300 import lib
    dev = torch.device("cuda", 0)
    nt, nph, mL = (int(x) for x in args.scan.split(","))
    w = W.plain_protein(seed=1, P=1)
    quats = W.euler_grid_quaternions(mL)
    D, R = nt * nph, quats.shape[0]
    ctx = lib.Context(0)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
    prot = lib.Protein(ctx, T(w.prot_xyz), T(w.prot_q), prm)
    lx, lq, tq = T(w.lig_xyz), T(w.lig_q), T(quats)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    scan = lambda: prot.ppiem_scan(lx, lq, tq, nt, nph)
    for _ in range(args.warmup):
        scan()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = lib.rs_stats_kernel_launches()
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            ev[i][0].record()
            out = scan()
            ev[i][1].record()
        torch.cuda.synchronize()
    launches = (lib.rs_stats_kernel_launches() - l0) // args.steps
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    lib.rs_timing_reset()
    lib.rs_timing_enable(2)
    for _ in range(2):
        scan()
    torch.cuda.synchronize()
    kernels = {k: round(v["ms"] / 2, 4) for k, v in
               sorted(lib.rs_timing_all().items(), key=lambda kv: -kv[1]["ms"])}
    lib.rs_timing_enable(0)
    o = {k: v.cpu().numpy() for k, v in out.items()}
    mins = np.nonzero(o["is_min"])[0]
    order = mins[np.argsort(o["E_best"][mins])]
    line = {"metric": "PPIEM pose scan: contact poses evaluated per second (A3 contact search + energy + minima)",
            "value": round(D * R / (ms / 1e3), 3), "unit": "poses/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
            "data": "synthetic", "dtype": "f64 contact offsets (f32 screen), f32-pair + bf16-slice energies",
            "config": {"workload": f"plain_protein (N=3000, L=50, n=1025, Tucker <= 20); {nt} x {nph} orbit "
                                   f"directions x {R} ZYZ Euler-grid self-rotations (m_L={mL})",
                       "poses": D * R, "l2": "flushed between steps (256 MiB write, outside the timed events)"},
            "result": {"feasible_fraction": float((o["flags"] == 0).mean()),
                       "contact_fraction": float(np.isfinite(o["s"]).mean()),
                       "local_minima": int(mins.size),
                       "lowest_minima": [{"direction": int(k), "E": float(o["E_best"][k]),
                                          "rotation": int(o["rot_best"][k])} for k in order[:5]]},
            "gpu_launches": int(launches), "clocks": clk.summary(), "kernels_ms_per_scan": kernels}
    if not args.no_cpu_baseline:
        import oracle as O
        rng = np.random.default_rng(0)
        pick = rng.choice(D * R, 64, replace=False)
        U = O.ppiem_directions(nt, nph)
        m = O.build_model(w.prot_xyz, w.prot_q, w.n, w.b, w.sigma, w.R_l, tucker_cap=w.tucker_cap)
        x_P = w.prot_xyz.mean(axis=0)
        t0 = time.perf_counter()
        s_ref = O.contact_offsets(w.prot_xyz, w.sigma, w.lig_xyz, quats[pick % R], x_P, U[pick // R])
        O.pose_energies(m, w.lig_xyz, w.lig_q, quats[pick % R], x_P + (s_ref + 1e-6 * w.sigma)[:, None] * U[pick // R])
        cs = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(pick.size / cs, 3), "unit": "poses/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": "64 random (direction, rotation) pairs of the scan: "
                                "brute-force contact + energy (the model build not timed)"}
    print(json.dumps(line), flush=True)
    prot.close()
    ctx.close()
    return 0


def run_localbox(args):
    """Scheme (C) of Sec. 3.2: the protein-scale potential re-truncated on a box around
    a cluster of poses outside the protein; energies of P poses in the box through the
    local handle, timed beside the global handle on the same poses."""
    import torch
    import workloads as W
    from paper_2510_26611_gb300 import lib
    dev = torch.device("cuda", 0)
    P = args.poses
    w = W.plain_protein(seed=1, P=1)
    rng = np.random.default_rng(21)
    c = np.array([0.0, 0.0, 28.0])
    half = 9.5
    r_l = float(np.linalg.norm(w.lig_xyz - w.lig_xyz.mean(axis=0), axis=1).max())
    spread = half - r_l - 0.5
    quat = W.shoemake_quaternions(rng, P)
    trans = c + rng.uniform(-spread, spread, size=(P, 3))
    ctx = lib.Context(0)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
    prot = lib.Protein(ctx, T(w.prot_xyz), T(w.prot_q), prm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loc = prot.local_box(c - half, c + half, eps=1e-7)
    build_ms = (time.perf_counter() - t0) * 1e3
    lx, lq, tq, tt = T(w.lig_xyz), T(w.lig_q), T(quat), T(trans)
    E = torch.empty(P, dtype=torch.float64, device=dev)
    F = torch.empty(P, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(h):
        for _ in range(args.warmup):
            lib.rs_energy_poses(ctx.handle, h, lx, lq, tq, tt, E_out=E, flags_out=F)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        l0 = lib.rs_stats_kernel_launches()
        with ClockSampler(0) as clk:
            for i in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                ev[i][0].record()
                lib.rs_energy_poses(ctx.handle, h, lx, lq, tq, tt, E_out=E, flags_out=F)
                ev[i][1].record()
            torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        return ms, E.cpu().numpy().copy(), F.cpu().numpy().copy(), clk.summary(), \
            (lib.rs_stats_kernel_launches() - l0) // args.steps

    ms_l, El, Fl, clocks, launches = timed(loc.handle)
    ms_g, Eg, Fg, _, _ = timed(prot.handle)
    lib.rs_timing_reset()
    lib.rs_timing_enable(2)
    for h in (loc.handle, prot.handle):
        for _ in range(2):
            lib.rs_energy_poses(ctx.handle, h, lx, lq, tq, tt, E_out=E, flags_out=F)
        torch.cuda.synchronize()
    kernels = {k: round(v["ms"] / 2, 4) for k, v in
               sorted(lib.rs_timing_all().items(), key=lambda kv: -kv[1]["ms"])}
    lib.rs_timing_enable(0)
    ok = (Fl & 2) == 0
    scale = np.maximum(np.abs(Eg), np.median(np.abs(Eg)))
    line = {"metric": "energies/s through a local-box handle (scheme C, Sec. 3.2)", "value": round(P / (ms_l / 1e3), 3),
            "unit": "poses/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_l, 4), "higher_is_better": True, "data": "synthetic",
            "dtype": "f32-pair + bf16-slice tensor-core evaluation",
            "config": {"workload": f"plain_protein (N=3000, L=50, n=1025, Tucker <= 20); box of half-width "
                                   f"{half} A around (0, 0, 28) A in the solvent beyond the protein's short axis; P poses with uniform "
                                   "rotations and centres within the box minus the ligand radius",
                       "poses": P, "eps": 1e-7, "l2": "flushed between steps (256 MiB write, outside the timed events)"},
            "global_handle": {"value": round(P / (ms_g / 1e3), 3), "ms_per_step": round(ms_g, 4)},
            "speedup_vs_global": round(ms_g / ms_l, 3),
            "ranks": {"global": list(prot.info["rank"]), "local": list(loc.info["rank"])},
            "local_build_ms": round(build_ms, 2),
            "max_rel_diff_to_global": float((np.abs(El - Eg) / scale)[ok].max()),
            "flags_equal_to_global": bool(np.array_equal(Fl, Fg)),
            "gpu_launches": int(launches), "clocks": clocks, "kernels_ms_local_then_global": kernels}
    print(json.dumps(line), flush=True)
    loc.close()
    prot.close()
    ctx.close()
    return 0


def run_complex(args):
    """Sec. 5.1, Eq. EnergySum_Mcomplex: the step's protein split into two molecules
    (by the sign of x), each built on its own; energies of P poses against the complex
    (one pose pass per molecule, summed on the device) timed beside the single molecule
    built on the union and beside the add-and-compressed sum of the two Tucker tensors
    (TEP step 4: one pose pass against one handle).  Then the Galerkin factors (Eq. galten) against collocation
    on the small canonical workload: energies/s of both and their difference."""
    import torch
    import workloads as W
    from paper_2510_26611_gb300 import lib
    dev = torch.device("cuda", 0)
    P = args.poses
    w, _ = workload(P, seed=1)
    ctx = lib.Context(0)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    prm = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
    side = w.prot_xyz[:, 0] >= 0
    mols = [lib.Protein(ctx, T(w.prot_xyz[sel]), T(w.prot_q[sel]), prm) for sel in (side, ~side)]
    union = lib.Protein(ctx, T(w.prot_xyz), T(w.prot_q), prm)
    lx, lq, tq, tt = T(w.lig_xyz), T(w.lig_q), T(w.quat), T(w.trans)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        l0 = lib.rs_stats_kernel_launches()
        with ClockSampler(0) as clk:
            for i in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                ev[i][0].record()
                out = fn()
                ev[i][1].record()
            torch.cuda.synchronize()
        return (sum(a.elapsed_time(b) for a, b in ev) / args.steps, out, clk.summary(),
                (lib.rs_stats_kernel_launches() - l0) // args.steps)

    ms_c, (Ec, Fc), clocks, launches = timed(
        lambda: lib.rs_energy_poses_complex(ctx.handle, [m.handle for m in mols], lx, lq, tq, tt))
    ms_u, (Eu, Fu), _, _ = timed(lambda: union.energies(lx, lq, tq, tt))
    # add-and-compress (TEP step 4): the two molecules' Tucker tensors summed and
    # re-truncated into one handle (host wall clock of the whole call: QR and HOSVD
    # on the host, cardinal basis, tables and the union's short range on the device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    acp = lib.Protein.add_compress(ctx, mols, w.tucker_cap)
    torch.cuda.synchronize()
    ms_build_ac = (time.perf_counter() - t0) * 1e3
    ms_a, (Ea, Fa), _, _ = timed(lambda: acp.energies(lx, lq, tq, tt))
    ac_info = acp.info
    acp.close()
    Ec, Eu, Fc, Fu = Ec.cpu().numpy(), Eu.cpu().numpy(), Fc.cpu().numpy(), Fu.cpu().numpy()
    Ea, Fa = Ea.cpu().numpy(), Fa.cpu().numpy()
    scale = np.maximum(np.abs(Eu), np.median(np.abs(Eu)))
    for m in mols:
        m.close()
    union.close()
    # Galerkin vs collocation (canonical, N=200, n=257; poses inside the protein's ball
    # so that the narrow long-range Gaussians, where cell averages differ, matter)
    ws = W.plain_small(P=20000)
    trans_in = W.ball_uniform(np.random.default_rng(4), ws.P, 12.0)
    res = {}
    for gal in (0, 1):
        pr = lib.Protein(ctx, T(ws.prot_xyz), T(ws.prot_q), lib.rs_params_default(
            n=ws.n, b=ws.b, sigma=ws.sigma, R_l=ws.R_l, tucker_cap=0, galerkin=gal))
        ms, (E, F), _, _ = timed(lambda: pr.energies(T(ws.lig_xyz), T(ws.lig_q), T(ws.quat), T(trans_in)))
        res[gal] = (ms, E.cpu().numpy())
        pr.close()
    dg = np.abs(res[1][1] - res[0][1]) / np.maximum(np.abs(res[0][1]), np.median(np.abs(res[0][1])))
    line = {"metric": "energies/s against a two-molecule complex (Eq. EnergySum_Mcomplex)",
            "value": round(P / (ms_c / 1e3), 3), "unit": "poses/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_c, 4), "higher_is_better": True, "data": "synthetic",
            "dtype": "f32-pair + bf16-slice tensor-core evaluation",
            "config": {"workload": "plain_protein split by the sign of x into two molecules of "
                                   f"{int(side.sum())} and {int((~side).sum())} atoms (each n=1025, Tucker <= 20); "
                                   "1e5 poses (L=50)", "poses": P,
                       "l2": "flushed between steps (256 MiB write, outside the timed events)"},
            "union_molecule": {"value": round(P / (ms_u / 1e3), 3), "ms_per_step": round(ms_u, 4)},
            # each molecule's Tucker form is truncated on its own (rank cap 20), so the
            # sum differs from the union's Tucker form by both truncation errors
            "max_rel_diff_complex_vs_union_tucker": float((np.abs(Ec - Eu) / scale).max()),
            "median_rel_diff_complex_vs_union_tucker": float(np.median(np.abs(Ec - Eu) / scale)),
            "flags_equal_complex_vs_union": bool(np.array_equal(Fc, Fu)),
            "add_compress": {"ranks": list(ac_info["rank"]), "sv_tail": [float(x) for x in ac_info["sv_tail"]],
                             "build_ms_wall": round(ms_build_ac, 3),
                             "poses_per_s": round(P / (ms_a / 1e3), 3), "ms_per_step": round(ms_a, 4),
                             "max_rel_diff_vs_complex": float((np.abs(Ea - Ec) / scale).max()),
                             "median_rel_diff_vs_complex": float(np.median(np.abs(Ea - Ec) / scale)),
                             "max_rel_diff_vs_union_tucker": float((np.abs(Ea - Eu) / scale).max()),
                             "flags_equal_vs_complex": bool(np.array_equal(Fa, Fc))},
            "galerkin": {"workload": "plain_small canonical (N=200, n=257, R = 4000), 2e4 poses with centres "
                                     "within 12 A of the protein's centre",
                         "collocation_poses_per_s": round(ws.P / (res[0][0] / 1e3), 3),
                         "galerkin_poses_per_s": round(ws.P / (res[1][0] / 1e3), 3),
                         "rel_diff_galerkin_vs_collocation": {"median": float(np.median(dg)), "max": float(dg.max())}},
            "gpu_launches": int(launches), "clocks": clocks}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# ------------------------------------------------------------------ serving mode
def _percentiles(x):
    x = np.asarray(x, dtype=np.float64)
    if x.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None, "count": 0}
    return {"p50_ms": round(float(np.percentile(x, 50)), 3), "p99_ms": round(float(np.percentile(x, 99)), 3),
            "mean_ms": round(float(x.mean()), 3), "count": int(x.size)}


def _serve_stream(args):
    import workloads as W
    rng = np.random.default_rng(11)
    pool = W.serve_pool(n_max=args.serve_n_max)
    arrivals = W.poisson_arrivals(rng, args.rate, args.duration)
    picks = rng.integers(0, len(pool), size=arrivals.size)
    return pool, arrivals, picks


def _serve_params(lib, e):
    return lib.rs_params_default(n=e["n"], b=e["b"], sigma=e["sigma"], R_l=e["R_l"],
                                 tucker_cap=e["tucker_cap"])


def _run_served(args, lib, pool, arrivals, picks):
    """Submits each request at its arrival time; a reaper thread collects results in
    submission order.  Latency = end - submit, from the library's own timestamps."""
    import queue
    import workloads as W
    knobs = {k: v for k, v in (("group_min_atoms", args.group_min_atoms),
                                ("group_atoms_per_cell", args.group_atoms_per_cell)) if v is not None}
    srv = lib.Server(0, **knobs)
    ids = queue.Queue()
    results = []

    def reaper():
        while True:
            item = ids.get()
            if item is None:
                return
            rid, k, cold = item
            res = srv.wait(rid, 600_000)
            results.append((k, cold, res["status"], res["t_submit_ns"], res["t_admit_ns"],
                            res["t_end_ns"], int(res["E"].shape[0])))

    # cold phase: the first request of every pool protein, all at once (builds the
    # resident factors); its latencies are the cold-start figures
    gen = np.random.default_rng(12)
    warm_ids = []
    tw = time.perf_counter()
    for e in pool:
        req = W.serve_request(gen, e)
        warm_ids.append((srv.submit(e["id"], e["xyz"], e["q"], _serve_params(lib, e), req["lig_xyz"],
                                    req["lig_q"], req["quat"], req["trans"]), req))
    cold = [srv.wait(rid, 3_600_000) for rid, _ in warm_ids]
    cold_wall = time.perf_counter() - tw
    cold_ms = [(r["t_end_ns"] - r["t_submit_ns"]) / 1e6 for r in cold if r["status"] == 0]
    th = threading.Thread(target=reaper, daemon=True)
    th.start()
    launches0 = lib.rs_stats_kernel_launches()
    st0 = srv.stats()
    t0 = time.perf_counter()
    for k, (ta, pi) in enumerate(zip(arrivals, picks)):
        e = pool[int(pi)]
        req = W.serve_request(gen, e)
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        rid = srv.submit(e["id"], e["xyz"], e["q"], _serve_params(lib, e), req["lig_xyz"],
                         req["lig_q"], req["quat"], req["trans"])
        ids.put((rid, k, False))
    ids.put(None)
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    st["launches"] -= st0["launches"]
    st["builds_in_stream"] = st["builds"] - st0["builds"]
    launches = lib.rs_stats_kernel_launches() - launches0
    srv.close()
    return results, wall, st, launches, cold_ms, cold_wall


def _run_plain(args, lib, pool, arrivals, picks):
    """The plain per-request path: one rs_energy_poses call (host buffers) per request
    in arrival order on one context, proteins built on first use and kept."""
    import workloads as W
    ctx = lib.Context(0)
    gen = np.random.default_rng(12)
    prots = {}
    for e in pool:  # the same cold phase: every protein built once, kept
        W.serve_request(gen, e)
        prots[e["id"]] = lib.Protein(ctx, e["xyz"], e["q"], _serve_params(lib, e))
    lat, lat_warm, poses = [], [], 0
    t0 = time.perf_counter()
    for ta, pi in zip(arrivals, picks):
        e = pool[int(pi)]
        req = W.serve_request(gen, e)
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        cold = e["id"] not in prots
        if cold:
            prots[e["id"]] = lib.Protein(ctx, e["xyz"], e["q"], _serve_params(lib, e))
        E, f = lib.rs_energy_poses(ctx.handle, prots[e["id"]].handle, req["lig_xyz"], req["lig_q"],
                                   req["quat"], req["trans"])
        done = time.perf_counter()
        ms = (done - (t0 + ta)) * 1e3
        lat.append(ms)
        if not cold:
            lat_warm.append(ms)
        poses += int(E.shape[0])
    wall = time.perf_counter() - t0
    for p in prots.values():
        p.close()
    ctx.close()
    return lat, lat_warm, poses, wall


def measure_serve(args) -> dict:
    """Serving (Poisson stream of docking requests against a pool of 64 proteins,
    grids n = 1025 ... 16385, 2048 poses per request): p50/p99 latency and poses/s of
    the serving loop beside the plain per-request path on the same stream."""
    from paper_2510_26611_gb300 import lib
    pool, arrivals, picks = _serve_stream(args)
    with ClockSampler(0) as clk:
        results, wall, st, launches, cold_ms, cold_wall = _run_served(args, lib, pool, arrivals, picks)
    clocks = clk.summary()
    ok = [r for r in results if r[2] == 0]
    lat = [(r[5] - r[3]) / 1e6 for r in ok]
    queue_ms = [(r[4] - r[3]) / 1e6 for r in ok]
    poses = sum(r[6] for r in ok)
    t_first = min(r[3] for r in results)
    t_last = max(r[5] for r in results)
    served = {"poses_per_s": round(poses / ((t_last - t_first) / 1e9), 1),
              "latency": _percentiles(lat), "admission_wait": _percentiles(queue_ms),
              "failed": len(results) - len(ok), "requests": len(results),
              "launches": st["launches"],
              "mean_requests_per_launch_incl_cold": round(st["mean_requests_per_launch"], 2),
              "builds_in_stream": st["builds_in_stream"], "evictions": st["evictions"],
              "resident_bytes": st["used_bytes"], "wall_s": round(wall, 2),
              "cold_start": {"latency": _percentiles(cold_ms), "builds": st["builds"],
                             "wall_s": round(cold_wall, 2)}}
    with ClockSampler(0) as clk_plain:
        plain_lat, plain_warm, plain_poses, plain_wall = _run_plain(args, lib, pool, arrivals, picks)
    plain = {"poses_per_s": round(plain_poses / plain_wall, 1), "latency": _percentiles(plain_lat),
             "wall_s": round(plain_wall, 2), "clocks": clk_plain.summary()}
    line = {"metric": "served p50/p99 latency and poses/s vs the plain per-request path",
            "value": served["poses_per_s"], "unit": "poses/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"serve: Poisson {args.rate:g} req/s for {args.duration:g} s; each "
                                   "request = a protein from a pool of 64 (N log-uniform "
                                   "[500, 20000], n by quintile of b in 1025..16385 capped at "
                                   f"{args.serve_n_max}, Tucker rank <= 20) + a new ligand "
                                   "(L uniform [10, 200]) + 2048 poses; admission by device "
                                   "memory, factors resident (a cold phase first builds every "
                                   "pool protein once; the stream is timed after it)",
                       "offered_poses_per_s":
                       round(args.rate * 2048, 1),
                       "grouping": {k: v for k, v in (("group_min_atoms", args.group_min_atoms),
                                                      ("group_atoms_per_cell", args.group_atoms_per_cell))
                                    if v is not None} or "library defaults"},
            "served": served, "plain": plain,
            "p50_ratio_plain_over_served": (round(plain["latency"]["p50_ms"] / served["latency"]["p50_ms"], 3)
                                            if served["latency"]["p50_ms"] and plain["latency"]["p50_ms"] else None),
            "p99_ratio_plain_over_served": (round(plain["latency"]["p99_ms"] / served["latency"]["p99_ms"], 3)
                                            if served["latency"]["p99_ms"] and plain["latency"]["p99_ms"] else None),
            "gpu_launches": int(launches), "clocks": clocks}
    return line


def run_serve(args):
    print(json.dumps(measure_serve(args)), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def job_step_time(t_local: float, world: int, device) -> float:
    """The whole job's time per step: the slowest rank's (MAX over ranks, returned on
    every rank).  Ranks evaluate their own poses against their own protein build with
    no data-path collective; this reduction and the barriers around the timed region
    are the only cross-rank operations."""
    import torch
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(poses_per_rank: int, world: int, seconds_per_step: float) -> float:
    """Poses per second of the whole job: every rank's poses over the slowest rank's time."""
    return world * poses_per_rank / seconds_per_step


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2510_26611_gb300 import lib

    P = args.poses
    w, rv = workload(P, seed=1 + rank)
    ctx = lib.Context(local)
    params = lib.rs_params_default(n=w.n, b=w.b, sigma=w.sigma, R_l=w.R_l, tucker_cap=w.tucker_cap)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    xyz, q = T(w.prot_xyz), T(w.prot_q)
    lx, lq = T(w.lig_xyz), T(w.lig_q)
    quat, trans, rvec = T(w.quat), T(w.trans), T(rv)
    E = torch.empty(P, dtype=torch.float64, device=dev)
    F = torch.empty(P, dtype=torch.uint8, device=dev)
    Eg = torch.empty(P, dtype=torch.float64, device=dev)
    Fg = torch.empty(P, dtype=torch.uint8, device=dev)
    gt = torch.empty((P, 3), dtype=torch.float64, device=dev)
    gw = torch.empty((P, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    h0 = lib.rs_build_protein(ctx.handle, xyz, q, params)
    ranks = lib.rs_protein_get_info(h0)["rank"]
    lib.rs_protein_free(h0)

    def step():
        h = lib.rs_build_protein(ctx.handle, xyz, q, params)
        lib.rs_energy_poses(ctx.handle, h, lx, lq, quat, trans, E_out=E, flags_out=F)
        lib.rs_energy_grad_poses(ctx.handle, h, lx, lq, rvec, trans, E_out=Eg, dE_dt=gt, dE_dw=gw,
                                 flags_out=Fg)
        lib.rs_protein_free(h)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    lib.rs_timing_reset()
    for g in (False, True):  # the atoms kernels count their work on the device
        lib.rs_diag_short_counts(local, grad=g, reset=True)
    lib.rs_timing_enable(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = lib.rs_stats_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()                       # L2 flush between steps (untimed)
            torch.cuda.synchronize()
            ev[i][0].record()
            step()
            ev[i][1].record()
        torch.cuda.synchronize()
        barrier()
    launches = lib.rs_stats_kernel_launches() - launches0
    lib.rs_timing_enable(0)
    timings = lib.rs_timing_all()
    short_work = {}
    for g, name in ((False, "k_sorted_atoms"), (True, "k_sorted_atoms_grad")):
        c = lib.rs_diag_short_counts(local, grad=g, reset=True)
        short_work[name] = c
        if name in timings:
            timings[name]["work"] = c["fp32_ops"]
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms_max = job_step_time(ms, world, dev)
    value = job_throughput(P, world, ms_max / 1e3)
    clocks = clk.summary()

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
        hx, hq, hlx, hlq = pin(w.prot_xyz), pin(w.prot_q), pin(w.lig_xyz), pin(w.lig_q)
        hquat, htr, hrv = pin(w.quat), pin(w.trans), pin(rv)
        hE = torch.empty(P, dtype=torch.float64).pin_memory()
        hF = torch.empty(P, dtype=torch.uint8).pin_memory()
        hEg = torch.empty(P, dtype=torch.float64).pin_memory()
        hFg = torch.empty(P, dtype=torch.uint8).pin_memory()
        hgt = torch.empty((P, 3), dtype=torch.float64).pin_memory()
        hgw = torch.empty((P, 3), dtype=torch.float64).pin_memory()

        def host_step():
            h = lib.rs_build_protein(ctx.handle, hx, hq, params)
            lib.rs_energy_poses(ctx.handle, h, hlx, hlq, hquat, htr, E_out=hE, flags_out=hF)
            lib.rs_energy_grad_poses(ctx.handle, h, hlx, hlq, hrv, htr, E_out=hEg, dE_dt=hgt,
                                     dE_dw=hgw, flags_out=hFg)
            lib.rs_protein_free(h)

        host_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        torch.cuda.synchronize()
        t_e2e = job_step_time((time.perf_counter() - t0) / args.steps, world, dev)
        L = w.L
        h2d = w.N * 32 + 2 * L * 32 + P * 32 + P * 24 + P * 24 + P * 24
        d2h = P * 8 + P + P * 8 + P * 48 + P
        e2e = {"value": round(job_throughput(P, world, t_e2e), 3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": round(1e3 * t_e2e, 3)}

    pose_atoms = {k: args.steps * P * w.L / max(timings[k]["launches"], 1)
                  for k in POSE_ATOM_KERNELS if k in timings}
    E_host = E.cpu().numpy()
    ctx.close()
    if rank == 0:
        pk = peaks(sm_count)
        top_name = max(timings.items(), key=lambda kv: kv[1]["ms"])[0] if timings else None
        rf = roofline(timings, pk, pose_atoms_per_launch=pose_atoms.get(top_name), ranks=ranks)
        cpu, errors = None, None
        if world == 1 and not args.no_cpu_baseline:
            fd, gpu_path = tempfile.mkstemp(suffix=".npy")
            os.close(fd)
            np.save(gpu_path, E_host[:ERROR_SAMPLE_POSES])
            try:
                cpu, errors = cpu_baseline(P, gpu_path)
            except Exception as e:  # report, do not hide
                cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                       "sample": f"failed: {type(e).__name__}: {str(e)[-300:]}"}
            finally:
                os.remove(gpu_path)
        extras = {}
        if world == 1 and not args.no_extras:
            for key, fn in (("served", measure_serve), ("batch", measure_batch), ("pgd", measure_pgd)):
                try:
                    extras[key] = fn(args)
                except Exception as e:  # report, do not hide
                    extras[key] = {"failed": f"{type(e).__name__}: {str(e)[-300:]}"}
        top = sorted(timings.values(), key=lambda r: -r["ms"])[:8]
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 build, f32-pair + bf16-slice tensor-core evaluation", "data": "synthetic",
                "config": {"workload": WORKLOAD, "poses_per_gpu": P, "ligand_atoms": w.L,
                           "protein_atoms": w.N, "n": w.n, "b": w.b, "tucker_cap": w.tucker_cap,
                           "l2": "flushed between steps (256 MiB write, outside the timed events)",
                           "parallelism": f"{world} independent ranks, poses split (no collective)"},
                "roofline": rf, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "roofline_pose_kernels": {k: roofline(timings, pk, k, pose_atoms.get(k), ranks)
                                          for k in POSE_ATOM_KERNELS if k in timings},
                "model_errors": errors,
                "short_range_work_per_step": {
                    k: {"atoms": v["atoms"] / args.steps, "candidates": v["candidates"] / args.steps,
                        "near_pairs": v["near"] / args.steps,
                        "fp32_gops": round(v["fp32_ops"] / args.steps / 1e9, 4)}
                    for k, v in short_work.items()},
                "clocks": clocks,
                "kernels_ms_per_step": {r["name"]: round(r["ms"] / args.steps, 4) for r in top}}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "build":
        return run_build(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "pgd":
        return run_pgd(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "fd":
        return run_fd(args)
    if args.mode == "ppiem":
        return run_ppiem(args)
    if args.mode == "localbox":
        return run_localbox(args)
    if args.mode == "complex":
        return run_complex(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
