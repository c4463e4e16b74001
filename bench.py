#!/usr/bin/env python3
"""Benchmark: SART reconstruction of the medium cylindrical workload on GB300.

Workload (one "step" = one whole reconstruction of one scan, every stage of the path):
  grid (N_h, N_theta, N_r) = (128, 512, 128), R 25 mm, H 50 mm; SOD 200, SDD 800 mm;
  180 views over 360 deg; 256 x 256 detector at 0.8 mm; seeded pose (|T| <= 2 mm,
  tilt <= 1 deg); five-shell part with eight inserts, one removed; Poisson counts at
  I0 = 1e4.  Step = re-pose the plan (ray tables) -> log transform of the counts ->
  20 SART sweeps (lambda 0.5) warm-started from the defect-free part's volume, with a
  4x weight inside the annulus r in [12, 18] mm.

Output: one JSON line (rank 0).  value = SART sweeps per second (whole job), with
GRays/s, the roofline of the dominant kernel, the CPU oracle baseline and the
end-to-end (host buffers) figure alongside.  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SART iters/sec and GRays/s at stated rel err; batched-serve vs plain scans/s, p99"
UNIT = "SART iters/s"
N_ITER = 20
# DRAM bytes (read + write) per launch of each kernel at the medium workload (one launch =
# one view), from one ncu capture of the same kernels on the medium grid and detector
# (k_rec_sart, k_update_rec4 and k_vox_sart1 on 8 of the 180 views; k_fp and k_bp, the
# two-launch form, from an earlier capture of the same walks).  k_rec_sart is the fused
# replay of the numerator form; the gather form's dominant kernel is k_vox_sart1.
TRAFFIC: dict = {"k_sart": 183.69e6, "k_update_nd4": 115.70e6, "k_fp": 73.27e6, "k_bp": 82.10e6,
                 "k_rec_sart": 181.85e6, "k_update_rec4": 122.61e6, "k_vox_sart1": 229.23e6}
# DRAM bytes per scan of the corner pass on Table 1 scans (FP16), from one ncu capture of
# 20 scans (profiles/pose_corners_table1.md); a launch's traffic scales with its scans.
TRAFFIC_PER_SCAN: dict = {"k_corners": 2.5122e9 / 20}
LAMBDA = 0.5
I0 = 1.0e4
CONFIG_MEDIUM = {
    "workload": "medium plain SART: grid (128,512,128) R25 H50, 180 views over 360 deg, 256x256 det "
                "0.8 mm, SOD 200 SDD 800, 20 sweeps lambda 0.5, warm start, ROI weights 4x (U8 class map), Poisson I0 1e4",
    "l2": "flushed (256 MB write) before every timed step",
    "data": "analytic line integrals of the continuous part (shells, inserts, one removed), Poisson counts",
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(rank: int = 0, views: int = 0):
    """The medium scan, its line integrals (analytic, of the continuous part with one insert
    removed), the defect-free warm start and the ROI weights.  views > 0: an evenly spaced
    selection of that many of its views (a small case of the same grid and detector for
    profiling captures)."""
    import dataclasses
    from paper_2005_11976_gb300 import synth
    rng = synth.rng_for("medium", rank)
    scan = synth.medium_scan(rng)
    if views > 0:
        scan = dataclasses.replace(scan, angles=scan.angles[::max(1, scan.n_proj // views)][:views])
    az = synth.insert_azimuths(rng)
    removed = int(rng.integers(8))
    p_part = synth.part_line_integrals(scan, az, removed=removed)   # the scanned part
    x_warm = synth.part_phantom(scan, az)                           # defect-free warm start
    w = synth.roi_weights(scan)
    return scan, p_part, x_warm, w, removed


def oracle_sample(scan, x_warm, counts_view, w, view: int):
    """FP64 oracle on one SART subset (one view) of the workload: (seconds, volume)."""
    import dataclasses
    import oracle
    s1 = dataclasses.replace(scan, angles=scan.angles[view:view + 1])
    o = oracle.Setup(**s1.fields())
    t0 = time.perf_counter()
    p = oracle.log_transform(counts_view, I0)
    x1 = oracle.sart(o, p, x0=x_warm, w=w, n_iter=1, lam=LAMBDA)
    return time.perf_counter() - t0, x1, o


def oracle_view_counts(scan, p_part, view: int):
    """Seeded Poisson counts of one view from the part's analytic line integrals (every input
    of an oracle run comes from synth)."""
    from paper_2005_11976_gb300 import synth
    return synth.poisson_counts(p_part[view:view + 1], I0, np.random.default_rng(5))


def run_reference(args):
    """The FP64 CPU oracle as it stands, timed on this host's cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    scan, p_part, x_warm, w, _ = workload(0)
    view = 37
    counts = oracle_view_counts(scan, p_part, view)
    times = []
    for k in range(args.warmup + args.steps):
        dt, _, _ = oracle_sample(scan, x_warm, counts, w, view)
        if k >= args.warmup:
            times.append(dt)
    t_subset = sum(times) / len(times)
    value = 1.0 / (t_subset * scan.n_proj)
    cores = oracle.num_threads()
    sample = f"one SART subset (view {view} of {scan.n_proj}) of the medium workload per step, scaled x{scan.n_proj}"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_subset * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(CONFIG_MEDIUM, sample=sample),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--eager", action="store_true",
                    help="eager launches with a CUDA event between kernels (default: one captured CUDA "
                         "graph per sweep, as cyl_sart_solve runs by default, timing events captured in it)")
    ap.add_argument("--workload", default="medium",
                    choices=["medium", "batched", "serving", "precision", "mtf", "pose", "table1", "table1_batch",
                             "phase", "l2ops"])
    ap.add_argument("--scans", type=int, default=0, help="batched/serving: number of scans")
    ap.add_argument("--no-batch-serve", action="store_true",
                    help="skip the bounded batched-vs-plain and served-vs-plain comparisons")
    ap.add_argument("--no-fused", action="store_true",
                    help="two launches per subset (projector, back-projector) instead of one")
    ap.add_argument("--views", type=int, default=0,
                    help="medium: run an evenly spaced selection of this many of the 180 views (a small "
                         "case for profiling captures; the JSON line then describes that case)")
    ap.add_argument("--record-form", type=int, default=1, choices=[1, 2],
                    help="medium: 1 back-projects by gathering per voxel from the records' transpose, "
                         "2 by replaying the records into a numerator")
    ap.add_argument("--record-runs", type=int, default=0,
                    help="medium: runs per ray of the stored segment records (0: the library's default)")
    ap.add_argument("--no-records", action="store_true",
                    help="medium: walk every ray in every subset instead of replaying the pose's "
                         "stored segment records")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "pose":
        return run_pose(args)
    if args.workload == "table1":
        return run_table1(args)
    if args.workload == "table1_batch":
        return run_table1_batch(args)
    if args.workload == "phase":
        return run_phase(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "mtf":
        return run_mtf(args)
    if args.workload == "l2ops":
        return run_l2ops(args)

    import torch
    from paper_2005_11976_gb300 import build as cbuild
    from paper_2005_11976_gb300 import cylct, replicas, synth

    rank, world, local = replicas.dist_env()
    torch.cuda.set_device(local)
    replicas.init("nccl", torch.device("cuda", local))
    if rank == 0 or not os.path.exists(cylct.LIB_PATH):
        cbuild.build()
    replicas.barrier()
    lib = cylct.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    scan, p_part, x_warm, w, removed = workload(rank, args.views)
    n_vox, n_pix = scan.n_vox, scan.det_w * scan.det_h
    plan = cylct.Plan(scan, device=local)
    pose = (scan.alpha, scan.beta, scan.gamma, scan.tx, scan.ty, scan.tz)

    # synthetic data: the part's analytic line integrals, Poisson counts drawn on the GPU
    # (seeded)
    p_clean = torch.from_numpy(p_part.astype(np.float32)).to(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(20051197 + rank)
    counts = torch.poisson(I0 * torch.exp(-p_clean), generator=gen)
    del p_clean
    x0 = torch.from_numpy(x_warm.astype(np.float32)).to(dev)
    wd = torch.from_numpy(_class_map(w)).to(dev)
    p = torch.empty_like(counts)
    x_out = torch.empty(scan.vol_shape, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    prm = cylct.sart_params(n_iter=N_ITER, lam=LAMBDA, use_graph=not args.eager, weight_dtype=cylct.CYL_U8)
    plan.cyl_plan_set_timing(True)
    plan.cyl_plan_set_fused(not args.no_fused)
    use_rec = not args.no_records and not args.no_fused
    if use_rec:
        plan.cyl_plan_set_records(args.record_form, args.record_runs, stream)
    rec_ready, rec_bytes, rec_gather, gather_bytes = plan.cyl_plan_records_full()

    def step(st):
        plan.cyl_plan_set_pose(pose, st)
        cylct.cyl_log_transform(counts, cylct.CYL_F32, I0, p, cylct.CYL_F32, counts.numel(), st)
        plan.cyl_sart_solve(p, cylct.CYL_F32, x0, wd, prm, x_out, cylct.CYL_F32, st)

    for _ in range(args.warmup):
        step(stream)
    torch.cuda.synchronize()

    # set-up cost of a pose: ray records and equal-step cuts of all views
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    plan.cyl_plan_set_pose(pose, stream)
    ev1.record(stream)
    ev1.synchronize()
    set_pose_ms = ev0.elapsed_time(ev1)

    # segments per view (algorithmic bytes of the projector)
    seg = torch.zeros(scan.n_proj, dtype=torch.int64, device=dev)
    plan.cyl_count_segments(0, scan.n_proj, seg, stream)
    torch.cuda.synchronize()
    seg = seg.cpu().numpy()

    clocks = ClockSampler(local)
    replicas.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    step_ms = []
    k_ms = [0.0, 0.0, 0.0]
    k_n = [0, 0, 0]
    for _ in range(args.steps):
        flush.fill_(1.0)                                # evict L2 between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for k in range(3):
            ms, n = plan.cyl_plan_kernel_time(k)
            k_ms[k] += ms
            k_n[k] += n
    torch.cuda.synchronize()
    replicas.barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    total_ms = replicas.max_over_ranks(float(sum(step_ms)), dev)
    value = replicas.whole_job_rate(args.steps * N_ITER, world, total_ms / 1e3)
    rays_per_sweep = 2 * scan.n_proj * n_pix         # forward + back-projected rays
    grays = world * args.steps * N_ITER * rays_per_sweep / (total_ms / 1e3) / 1e9

    # --- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h_counts = counts.cpu().pin_memory()
        h_out = torch.empty(scan.vol_shape, dtype=torch.float32).pin_memory()

        def e2e_step(st):
            # every transfer through the C ABI: the log transform reads the pinned host counts
            # (device-addressable), the solve writes its result to the pinned host volume
            plan.cyl_plan_set_pose(pose, st)
            cylct.cyl_log_transform(h_counts, cylct.CYL_F32, I0, p, cylct.CYL_F32,
                                    counts.numel(), st)
            plan.cyl_sart_solve(p, cylct.CYL_F32, x0, wd, prm, h_out, cylct.CYL_F32, st)

        e2e_step(stream)
        torch.cuda.synchronize()
        replicas.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step(stream)
        torch.cuda.synchronize()
        e2e_t = replicas.max_over_ranks(time.perf_counter() - t0, dev)
        replicas.barrier()
        e2e = {"value": replicas.whole_job_rate(args.steps * N_ITER, world, e2e_t), "unit": UNIT,
               "h2d_bytes_per_step": int(counts.numel() * 4),
               "d2h_bytes_per_step": int(n_vox * 4)}

    # --- roofline of the dominant kernel, on the segment-touch byte model of the path's
    # specification: forward S b_v + H W (b_s + 4); back-projection and update together
    # S 4 + 2 V_hit b_v + V_hit b_w (V_hit = V: every voxel of the grid is crossed by some
    # ray of a medium view).  One launch of every kernel covers one view (one subset).
    hbm, peak_kind = peaks()
    roof = None
    if k_n[0] and k_n[2]:
        S = float(seg.sum()) / scan.n_proj           # segments per view (= per launch)
        b_v, b_s, b_w = 4, 4, 1                      # FP32 volume and data, U8 class map
        fwd = S * b_v + n_pix * (b_s + 4)
        back = S * 4                                 # the residual carried to every segment
        upd = 2 * n_vox * b_v + n_vox * b_w          # x read and written, w read
        avg_ms = [k_ms[k] / k_n[k] if k_n[k] else 0.0 for k in range(3)]
        t_view = sum(avg_ms) / 1e3
        if args.no_fused:
            names = ["forward projection (k_fp)", "back-projection into (num, den) (k_bp)",
                     "SART voxel update (k_update_nd4)"]
            per = [fwd, back, upd]
        elif rec_ready and rec_gather:
            names = ["projection and residual from the stored segment records (k_rec_sart, forward replay)",
                     None, "back-projection gathered per voxel with its column sums and the update (k_vox_sart1)"]
            per = [fwd, 0.0, back + upd]
        elif rec_ready:
            names = ["projection, residual and back-projection from the stored segment records (k_rec_sart)",
                     None, "SART voxel update with the pose's column sums (k_update_rec4)"]
            per = [fwd + back, 0.0, upd]
        else:
            names = ["projection, residual and back-projection, one walk (k_sart)", None,
                     "SART voxel update (k_update_nd4)"]
            per = [fwd + back, 0.0, upd]
        ach = [per[k] / (avg_ms[k] / 1e3) / 1e9 if k_n[k] else 0.0 for k in range(3)]
        dom = int(np.argmax(k_ms))
        kernel = names[dom].split("(")[-1][:-1]
        # the builder's own per-kernel model: what the kernels move as built (48-byte ray
        # records, the spare accumulator cleared, the packed 8-byte (num, den) reduction)
        own = {"forward": S * 4 + n_pix * (48 + 4) + n_vox * 8,
               "back": S * 8 + n_pix * (48 + 4 + 4),
               "update": n_vox * (8 + 4 + 4 + 1)}
        # compulsory model: every array of a subset once (x read by the projector, read and
        # written by the update; w; p, q and the residual)
        comp = 3 * n_vox * 4 + n_vox * 1 + 3 * n_pix * 4
        roof = {"bound": "hbm", "achieved": ach[dom], "peak": hbm, "unit": "GB/s",
                "frac": ach[dom] / hbm, "traffic": TRAFFIC.get(kernel),
                "kernel": names[dom], "peak_source": peak_kind, "model": "segment-touch (path specification)",
                "algorithmic_bytes_per_launch": per[dom],
                "units_per_launch": "one view: %d rays, %.4g segments" % (n_pix, S),
                "path_per_view": {"bytes": fwd + back + upd, "ms": t_view * 1e3,
                                  "achieved": (fwd + back + upd) / t_view / 1e9,
                                  "frac": (fwd + back + upd) / t_view / 1e9 / hbm},
                "forward": {"bytes": fwd}, "back_and_update": {"bytes": back + upd},
                "kernel_ms_avg": {names[k]: avg_ms[k] for k in range(3) if names[k]},
                "kernel_gbs": {names[k]: ach[k] for k in range(3) if names[k]},
                "kernel_frac": {names[k]: ach[k] / hbm for k in range(3) if names[k]},
                "kernel_share": {names[k]: k_ms[k] / sum(k_ms) for k in range(3) if names[k]},
                "segments_per_view": S,
                "compulsory_model": {"bytes_per_subset": comp, "achieved": comp / t_view / 1e9,
                                     "frac": comp / t_view / 1e9 / hbm, "unit": "GB/s"},
                "own_model_bytes_per_view": own}
        if args.no_fused:
            t_fp, t_bu = avg_ms[0] / 1e3, (avg_ms[1] + avg_ms[2]) / 1e3
            roof["forward"].update(achieved=fwd / t_fp / 1e9, frac=fwd / t_fp / 1e9 / hbm)
            roof["back_and_update"].update(achieved=(back + upd) / t_bu / 1e9,
                                           frac=(back + upd) / t_bu / 1e9 / hbm)

    # --- CPU oracle on a bounded sample, and a live parity check on that sample
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import dataclasses
        import oracle
        oracle.build()
        view = min(37, scan.n_proj - 1)
        counts_v = oracle_view_counts(scan, p_part, view)
        oracle_sample(scan, x_warm, counts_v, w, view)          # warm-up (pages, threads)
        runs = [oracle_sample(scan, x_warm, counts_v, w, view) for _ in range(3)]
        dt, x1_or = sum(r[0] for r in runs) / len(runs), runs[-1][1]
        cores = oracle.num_threads()
        oracle.set_num_threads(1)
        dt1, _, _ = oracle_sample(scan, x_warm, counts_v, w, view)
        oracle.set_num_threads(cores)
        cpu = {"value": 1.0 / (dt * scan.n_proj), "unit": UNIT, "cores": cores,
               "kind": "oracle",
               "sample": f"one SART subset (view {view} of {scan.n_proj}) of the medium workload, "
                         f"{dt:.2f} s on {cores} threads (mean of 3 after a warm-up), {dt1:.2f} s on one; "
                         f"scaled x{scan.n_proj}",
               "value_one_thread": 1.0 / (dt1 * scan.n_proj)}
        s1 = dataclasses.replace(scan, angles=scan.angles[view:view + 1])
        with cylct.Plan(s1, device=local) as p1:
            cv = torch.from_numpy(counts_v.astype(np.float32)).to(dev)
            pv = torch.empty_like(cv)
            cylct.cyl_log_transform(cv, cylct.CYL_F32, I0, pv, cylct.CYL_F32, n_pix, stream)
            xg = torch.empty_like(x_out)
            p1.cyl_sart_solve(pv, cylct.CYL_F32, x0, wd, cylct.sart_params(n_iter=1, lam=LAMBDA, weight_dtype=cylct.CYL_U8),
                              xg, cylct.CYL_F32, stream)
            torch.cuda.synchronize()
            xg = xg.cpu().numpy().astype(np.float64)
        parity = float(np.linalg.norm(xg - x1_or) / np.linalg.norm(x1_or))

    # --- the metric's second half on the same GPU, bounded: batched vs plain scans/s, and
    # served vs plain scans/s with p50 / p99 latency on a stream the GPU sustains
    batched = serving = None
    if rank == 0 and world == 1 and not args.no_batch_serve:
        plan.cyl_plan_set_timing(False)
        batched = {k: v for k, v in batched_compare(torch, cylct, 16).items() if k != "per_scan_rel_err"}
        # at the configured 20 scans/s the GPU saturates (throughput); at 3 scans/s it keeps up
        # and the queue stays short (latency); the large part type is left to --workload serving
        serving = {}
        for key, rate in (("saturated", 20.0), ("sustained", 3.0)):
            r = serving_compare(torch, cylct, 24, rate, 60.0, ("small", "medium"))
            serving[key] = {k: v for k, v in r.items() if k not in ("latencies_s", "plain_latencies_s")}

    # per step: ray records + cuts (set_pose, with the segment records' launches), log,
    # weight max + scale, and per subset the projector, the back-projector and the update
    per_pose = 0
    if rec_ready:   # rows, scan, record walk; then the transpose (count, three scan passes,
        # base, fill per view) or the column sums (two per view)
        per_pose = 3 + (6 * scan.n_proj if rec_gather else 2 * scan.n_proj)
    n_launch = args.steps * (2 + per_pose + 1 + 2 + N_ITER * scan.n_proj * (3 if args.no_fused else 2))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(CONFIG_MEDIUM,
                       launch="one captured CUDA graph per sweep, CUDA events captured between its "
                              "kernels (kernel times: the last sweep of every timed step)" if not args.eager
                       else "eager, a CUDA event between launches",
                       parallelism="replicas" if world > 1 else "single GPU",
                       **({"views": f"{scan.n_proj} evenly spaced of the 180 views (profiling case)"}
                          if args.views else {})),
        "grays_per_s": grays, "rel_err_vs_oracle_one_subset": parity, "set_pose_ms": set_pose_ms,
        "segment_records": {"used": rec_ready, "bytes": rec_bytes,
                            "bytes_per_view": rec_bytes / scan.n_proj,
                            "gather_per_voxel": rec_gather, "transpose_bytes": gather_bytes,
                            "note": "each pose's pieces written once at set-up (inside every timed step) "
                                    "and replayed by the subsets, read twice per subset (forward and back)"}
                           if use_rec else {"used": False},
        "rel_err_bound": "<=1e-5 rel L2 per projection and per iterate (tests)",
        "wall_s_timed": t_wall, "clocks": clk, "gpu_launches": n_launch,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "batched_vs_plain": batched, "serving_vs_plain": serving,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0



# ------------------------------------------------------------------ batched / serving

def _gpu_setup():
    """This rank's GPU (the local rank under torchrun), its process group, and the library
    (built by rank 0)."""
    import torch
    from paper_2005_11976_gb300 import build as cbuild
    from paper_2005_11976_gb300 import cylct, replicas
    rank, world, local = replicas.dist_env()
    torch.cuda.set_device(local)
    replicas.init("nccl", torch.device("cuda", local))
    if rank == 0 or not os.path.exists(cylct.LIB_PATH):
        cbuild.build()
    replicas.barrier()
    cylct.load()
    return torch, cylct


def _part_data(scan, rng):
    """Warm start (defect-free part) and a scanned part with one insert removed."""
    from paper_2005_11976_gb300 import synth
    az = synth.insert_azimuths(rng)
    return synth.part_phantom(scan, az), synth.part_phantom(scan, az, removed=int(rng.integers(8)))


def _class_map(w):
    """The ROI weight map (weights 1 and 4) as a U8 class map: one byte per voxel."""
    v = np.rint(w)
    assert np.array_equal(v, w) and v.min() >= 0 and v.max() <= 255
    return v.astype(np.uint8)


def _sinogram(torch, cylct, plan, scan, x_part, i0, seed, dtype):
    """Line integrals of x_part projected on the GPU with Poisson counts at I0."""
    dev = torch.device("cuda")
    xp = torch.from_numpy(x_part.astype(np.float32)).to(dev)
    p = torch.empty(scan.sino_shape, device=dev)
    plan.cyl_project(xp, cylct.CYL_F32, 0, scan.n_proj, p, cylct.CYL_F32)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    counts = torch.poisson(i0 * torch.exp(-p), generator=gen)
    out = torch.empty(scan.sino_shape, dtype={0: torch.float32, 1: torch.float16, 2: torch.bfloat16}[dtype],
                      device=dev)
    cylct.cyl_log_transform(counts, cylct.CYL_F32, i0, out, dtype, counts.numel())
    return out


def batched_compare(torch, cylct, n, ids=None):
    """Scans `ids` (default: all) of a batch of n scans of one part type (own pose, N_p in
    {60, 90, 120, 180}): one batched graph launch vs one cyl_sart_solve per scan, 10 sweeps
    each, FP32.  Returns the figures of this process's scans."""
    from paper_2005_11976_gb300 import replicas, synth
    ids = list(range(n)) if ids is None else list(ids)
    scans = [synth.batched_scans(n)[i] for i in ids]
    n = len(scans)                     # this process's scans
    rng = synth.rng_for("batched", 1000)
    x_warm, x_part = _part_data(scans[0], rng)
    w = synth.roi_weights(scans[0])
    dev = torch.device("cuda")
    x0 = torch.from_numpy(x_warm.astype(np.float32)).to(dev)
    wd = torch.from_numpy(_class_map(w)).to(dev)
    plans = [cylct.Plan(s) for s in scans]
    sinos = [_sinogram(torch, cylct, plans[i], s, x_part, I0, 100 + i, cylct.CYL_F32)
             for i, s in enumerate(scans)]
    outs_b = [torch.empty(s.vol_shape, device=dev) for s in scans]
    outs_p = [torch.empty(s.vol_shape, device=dev) for s in scans]
    prm = cylct.sart_params(n_iter=10, lam=LAMBDA, weight_dtype=cylct.CYL_U8)
    # the batch autotuner times round 0 for every piece setting (the batch uses plans[0]'s)
    cylct.cyl_sart_tune_batch(plans, sinos, cylct.CYL_F32, [x0] * n, [wd] * n, prm, outs_b, cylct.CYL_F32)
    pieces = plans[0].cyl_plan_get_pieces()
    # warm-up: one small batched and one plain solve
    cylct.cyl_sart_solve_batch(plans[:2], sinos[:2], cylct.CYL_F32, [x0, x0], [wd, wd],
                               cylct.sart_params(n_iter=1, lam=LAMBDA, weight_dtype=cylct.CYL_U8), outs_b[:2], cylct.CYL_F32)
    plans[0].cyl_sart_solve(sinos[0], cylct.CYL_F32, x0, wd, cylct.sart_params(n_iter=1, lam=LAMBDA, weight_dtype=cylct.CYL_U8),
                            outs_p[0], cylct.CYL_F32)
    torch.cuda.synchronize()
    replicas.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    cylct.cyl_sart_solve_batch(plans, sinos, cylct.CYL_F32, [x0] * n, [wd] * n, prm, outs_b,
                               cylct.CYL_F32)
    e1.record()
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    e0.record()
    for i in range(n):
        plans[i].cyl_sart_solve(sinos[i], cylct.CYL_F32, x0, wd, prm, outs_p[i], cylct.CYL_F32)
    e1.record()
    e1.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    # plain with stored segment records: each scan writes its records and column sums, is
    # solved, and frees them (all scans' records at once would not fit); the record
    # set-up is inside the timed region
    outs_r = [torch.empty(s.vol_shape, device=dev) for s in scans]
    e0.record()
    for i in range(n):
        plans[i].cyl_plan_set_records(1)
        plans[i].cyl_sart_solve(sinos[i], cylct.CYL_F32, x0, wd, prm, outs_r[i], cylct.CYL_F32)
        plans[i].cyl_plan_set_records(0)
    e1.record()
    e1.synchronize()
    t_rec = e0.elapsed_time(e1) / 1e3
    err_rec = max(float((outs_r[i] - outs_p[i]).norm() / outs_p[i].norm()) for i in range(n))
    del outs_r
    errs = [float((outs_b[i] - outs_p[i]).norm() / outs_p[i].norm()) for i in range(n)]
    err = max(errs)
    views = sum(s.n_proj for s in scans)
    for p in plans:
        p.close()
    return {"scans": n, "views": views, "per_scan_rel_err": errs, "batched_scans_per_s": n / t_batch, "plain_scans_per_s": n / t_plain,
            "batched_over_plain": t_plain / t_batch, "max_rel_err_batched_vs_plain": err,
            "batched_s": t_batch, "plain_s": t_plain,
            "plain_records_scans_per_s": n / t_rec, "batched_over_plain_records": t_rec / t_batch,
            "max_rel_err_plain_records_vs_plain": err_rec,
            "pieces_per_ray_tuned": {"projector": pieces[0], "back_projector": pieces[1]},
            "sart_iters_per_s_batched": n * 10 / t_batch,
            "grays_per_s_batched": 2 * 10 * views * scans[0].det_w * scans[0].det_h / t_batch / 1e9,
            "workload": f"{n} scans of one part, grid (128,512,128), 256x256 det, N_p in {{60,90,120,180}} "
                        f"({views} views), |T|<=5 mm, tilt<=3 deg, 10 sweeps, shared warm start, ROI weights "
                        "(U8 class map), FP32; one CUDA graph (batched) vs one cyl_sart_solve graph per scan (plain)"}


def run_batched(args):
    """64 scans of one part type (own pose, N_p in {60, 90, 120, 180}) reconstructed by one
    batched graph launch vs one cyl_sart_solve per scan, 10 sweeps each, FP32.  Under
    torchrun the batch is sharded by scan over the ranks (no data-path collective); the
    rates are all scans over the slowest rank's time, and rank 0 gathers the per-scan
    batched-vs-plain errors in the batch's order."""
    torch, cylct = _gpu_setup()
    from paper_2005_11976_gb300 import replicas
    rank, world, local = replicas.dist_env()
    n = args.scans or 64
    clocks = ClockSampler(local)
    clocks.start()
    r = batched_compare(torch, cylct, n, replicas.shard(n, rank, world))
    clk = clocks.stop()
    t_b = replicas.max_over_ranks(r["batched_s"], torch.device("cuda", local))
    t_p = replicas.max_over_ranks(r["plain_s"], torch.device("cuda", local))
    errs = replicas.gather_ordered(r["per_scan_rel_err"], n, rank, world)
    if rank == 0:
        line = {
            "metric": METRIC, "value": n / t_b, "unit": "scans/s", "n_gpus": world, "steps": 1,
            "warmup": 1, "ms_per_step": t_b * 1e3, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched: " + r["workload"].replace(f"{r['scans']} scans", f"{n} scans"),
                       "parallelism": f"scan-sharded over {world} GPUs" if world > 1 else "single GPU"},
            "clocks": clk, "plain_scans_per_s": n / t_p, "batched_over_plain": t_p / t_b,
            "max_rel_err_batched_vs_plain": max(errs), "per_scan_rel_err_batched_vs_plain": errs,
            "pieces_per_ray_tuned": r["pieces_per_ray_tuned"],
        }
        print(json.dumps(line), flush=True)
    return 0


def run_table1(args):
    """SART on the paper's own reconstruction workload (Sec. 3.3 with Table 1): grid
    (N_h, N_theta, N_r) = (240, 40, 60) over the 64 mm x R8 part, 21 projections over
    200 deg on the 1944 x 1536 panel (0.0748 mm), SOD 679, SDD 791.  Plain SART from the
    warm start, and SART with the weighted back-projection (weight 4 in an annulus), 10
    sweeps each, FP32.  The paper reports 0.30 s (plain) and 0.52 s (weighted) for its
    reconstructions, iteration count unstated."""
    import dataclasses
    torch, cylct = _gpu_setup()
    from paper_2005_11976_gb300 import synth
    dev = torch.device("cuda")
    sweeps = 10
    scan = synth.table1_scan(grid=(240, 40, 60))
    rng = synth.rng_for("table1", 0)
    scan.alpha, scan.beta, scan.gamma, scan.tx, scan.ty, scan.tz = synth.seeded_pose(rng, 2.0, 1.0)
    x_warm, x_part = _part_data(scan, rng)
    w = synth.roi_weights(scan)
    plan = cylct.Plan(scan)
    sino = _sinogram(torch, cylct, plan, scan, x_part, I0, 77, cylct.CYL_F32)
    x0 = torch.from_numpy(x_warm.astype(np.float32)).to(dev)
    wd = torch.from_numpy(_class_map(w)).to(dev)
    out = torch.empty(scan.vol_shape, device=dev)
    plain = cylct.sart_params(n_iter=sweeps, lam=LAMBDA, weight_dtype=cylct.CYL_U8)
    plan.cyl_plan_tune()                       # pieces per ray for this plan (times view 0)
    pieces = plan.cyl_plan_get_pieces()
    for _ in range(max(3, args.warmup)):
        plan.cyl_sart_solve(sino, cylct.CYL_F32, x0, None, cylct.sart_params(n_iter=1, lam=LAMBDA), out,
                            cylct.CYL_F32)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t = {"plain": [], "weighted": []}
    for _ in range(args.steps):
        for kind, wt in (("plain", None), ("weighted", wd)):
            e0.record()
            plan.cyl_sart_solve(sino, cylct.CYL_F32, x0, wt, plain, out, cylct.CYL_F32)
            e1.record()
            e1.synchronize()
            t[kind].append(e0.elapsed_time(e1) / 1e3)
    clk = clocks.stop()
    tp, tw = float(np.mean(t["plain"])), float(np.mean(t["weighted"]))
    # segments of one sweep, for GRays/s and the walk's rate
    cnt = torch.empty(scan.n_proj, dtype=torch.int64, device=dev)
    plan.cyl_count_segments(0, scan.n_proj, cnt)
    segs = int(cnt.sum().item())
    hit = torch.empty(scan.sino_shape, device=dev)
    plan.cyl_row_sums(0, scan.n_proj, hit)
    rays_hit = int((hit > 0).sum().item())
    cpu = parity = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        view = 10
        counts_v = oracle_view_counts(scan, p_part, view)
        dt, x1_or, _ = oracle_sample(scan, x_warm, counts_v, w, view)
        cpu = {"value": 1.0 / (dt * scan.n_proj), "unit": "sweeps/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"one SART subset (view {view} of 21), {dt:.2f} s, scaled x21"}
        s1 = dataclasses.replace(scan, angles=scan.angles[view:view + 1])
        with cylct.Plan(s1) as p1:
            cv = torch.from_numpy(counts_v.astype(np.float32)).to(dev)
            pv = torch.empty_like(cv)
            cylct.cyl_log_transform(cv, cylct.CYL_F32, I0, pv, cylct.CYL_F32, cv.numel())
            xg = torch.empty_like(out)
            p1.cyl_sart_solve(pv, cylct.CYL_F32, x0, wd, cylct.sart_params(n_iter=1, lam=LAMBDA, weight_dtype=cylct.CYL_U8), xg, cylct.CYL_F32)
            torch.cuda.synchronize()
            xg = xg.cpu().numpy().astype(np.float64)
        parity = float(np.linalg.norm(xg - x1_or) / np.linalg.norm(x1_or))
    n_pix = scan.det_w * scan.det_h
    plan_bytes = plan.sizes()[3]
    line = {
        "metric": "SART sweeps/s on the paper's Table 1 reconstruction workload", "value": sweeps / tp,
        "unit": "SART iters/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": (tp + tw) * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "table1: grid (240,40,60) R8 H64, 21 views over 200 deg, 1944x1536 at 0.0748 mm, "
                               "SOD 679 SDD 791, shells + 8 inserts (one removed), Poisson I0 1e4, warm start, "
                               "10 sweeps plain and 10 weighted (4x annulus)",
                   "l2": "not flushed; each sweep reads the records and cuts of the 5.3 M rays that meet "
                         "the grid (422 MB), more than L2"},
        "baseline_note": "the paper: 0.30 s plain, 0.52 s weighted per reconstruction, iterations unstated",
        "s_per_sweep": {"plain": tp / sweeps, "weighted": tw / sweeps},
        "s_per_10_sweeps": {"plain": tp, "weighted": tw},
        "weighted_over_plain": tw / tp,
        "rays_per_sweep": n_pix * scan.n_proj, "rays_hitting_the_grid": rays_hit, "segments_per_sweep": segs,
        "grays_per_s": 2 * sweeps * n_pix * scan.n_proj / tp / 1e9,
        "rel_err_vs_oracle_one_subset": parity, "plan_device_bytes": plan_bytes, "clocks": clk,
        "pieces_per_ray_tuned": {"projector": pieces[0], "back_projector": pieces[1]},
        # per step: projector, back-projector and update per view and sweep in both solves,
        # and the weight maximum and scale of the weighted one
        "gpu_launches": args.steps * (2 * sweeps * scan.n_proj * 3 + 2),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def run_table1_batch(args):
    """The in-line batch of Sec. 2.4 on Table 1's acquisition: 16 scans of the part (grid
    (240, 40, 60), 21 views over 200 deg, 1944 x 1536 panel), each at its own seeded pose,
    shared warm start, 10 sweeps, FP32: one batched graph (autotuned pieces; the scans'
    rays that meet the grid listed) vs one cyl_sart_solve per scan."""
    torch, cylct = _gpu_setup()
    import dataclasses
    from paper_2005_11976_gb300 import synth
    dev = torch.device("cuda")
    n = args.scans or 16
    base = synth.table1_scan(grid=(240, 40, 60))
    rng = synth.rng_for("table1", 100)
    x_warm, x_part = _part_data(base, rng)
    scans = []
    for i in range(n):
        s = dataclasses.replace(base)
        s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz = synth.seeded_pose(rng, 2.0, 1.0)
        scans.append(s)
    plans = [cylct.Plan(s) for s in scans]
    sinos = [_sinogram(torch, cylct, plans[i], s, x_part, I0, 300 + i, cylct.CYL_F32) for i, s in enumerate(scans)]
    x0 = torch.from_numpy(x_warm.astype(np.float32)).to(dev)
    outs_b = [torch.empty(base.vol_shape, device=dev) for _ in range(n)]
    outs_p = [torch.empty(base.vol_shape, device=dev) for _ in range(n)]
    prm = cylct.sart_params(n_iter=10, lam=LAMBDA)
    cylct.cyl_sart_tune_batch(plans, sinos, cylct.CYL_F32, [x0] * n, None, prm, outs_b, cylct.CYL_F32)
    pieces = plans[0].cyl_plan_get_pieces()
    cylct.cyl_sart_solve_batch(plans[:2], sinos[:2], cylct.CYL_F32, [x0, x0], None,
                               cylct.sart_params(n_iter=1, lam=LAMBDA), outs_b[:2], cylct.CYL_F32)
    plans[0].cyl_sart_solve(sinos[0], cylct.CYL_F32, x0, None, cylct.sart_params(n_iter=1, lam=LAMBDA),
                            outs_p[0], cylct.CYL_F32)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    cylct.cyl_sart_solve_batch(plans, sinos, cylct.CYL_F32, [x0] * n, None, prm, outs_b, cylct.CYL_F32)
    e1.record()
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    e0.record()
    for i in range(n):
        plans[i].cyl_sart_solve(sinos[i], cylct.CYL_F32, x0, None, prm, outs_p[i], cylct.CYL_F32)
    e1.record()
    e1.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    clk = clocks.stop()
    err = max(float((outs_b[i] - outs_p[i]).norm() / outs_p[i].norm()) for i in range(n))
    line = {
        "metric": "SART scans/s on the paper's in-line batch (Table 1 acquisition)", "value": n / t_batch,
        "unit": "scans/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": t_batch * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"table1_batch: {n} scans, grid (240,40,60) R8 H64, 21 views over 200 deg, "
                               "1944x1536 at 0.0748 mm, SOD 679 SDD 791, seeded poses (|T| <= 2 mm, tilt <= 1 deg), "
                               "shared warm start, Poisson I0 1e4, 10 sweeps",
                   "launch": "one CUDA graph (batched) vs one cyl_sart_solve graph per scan (plain)"},
        "pieces_per_ray_tuned": {"projector": pieces[0], "back_projector": pieces[1]},
        "plain_scans_per_s": n / t_plain, "batched_over_plain": t_plain / t_batch,
        "max_rel_err_batched_vs_plain": err, "ms_per_scan_batched": t_batch * 1e3 / n,
        "baseline_note": "the paper: 0.30 s per reconstruction (plain), iterations and hardware unstated",
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    return 0


def run_phase(args):
    """Pose and azimuthal phase (Sec. 2.1, Eq. 3-5) of Table 1 scans: parts that carry one
    off-axis metal pin (a tube 64 mm x R8 / R3, pin r 0.8 mm at r 5.5 mm), each at a
    seeded pose with a seeded spin gamma; 21 projections over 200 deg on the 1944 x 1536
    panel (0.0748 mm), Poisson I0 4e4, FP16.  Per scan: the pose estimate, the plan
    re-posed with the estimated axis and gamma = 0, and cyl_estimate_gamma against the
    part's template (the pin at azimuth 0), three passes.  Reports the time per scan and
    the gamma error against the truth."""
    torch, cylct = _gpu_setup()
    from paper_2005_11976_gb300 import synth
    dev = torch.device("cuda")
    n_parts = args.scans or 20
    base = synth.table1_scan(grid=(64, 96, 32))
    x_t = synth.pinned_tube(base)
    xt = torch.from_numpy(x_t.astype(np.float32)).to(dev)
    rng = synth.rng_for("phase", 0)
    truth = [(float(rng.uniform(0, 2 * math.pi)), math.radians(float(rng.uniform(0.5, 3.0))),
              float(rng.uniform(-math.pi, math.pi)), *[float(v) for v in rng.uniform(-2.0, 2.0, 3)])
             for _ in range(n_parts)]
    i0_p = 4.0e4
    gen = torch.Generator(device=dev)
    gen.manual_seed(777)
    plan = cylct.Plan(base)
    p32 = torch.empty(base.sino_shape, device=dev)
    sinos = []
    for t in truth:
        plan.cyl_plan_set_pose(t)
        plan.cyl_project(xt, cylct.CYL_F32, 0, base.n_proj, p32, cylct.CYL_F32)
        counts = torch.poisson(i0_p * torch.exp(-p32), generator=gen)
        sv = torch.empty(base.sino_shape, dtype=torch.float16, device=dev)
        cylct.cyl_log_transform(counts, cylct.CYL_F32, i0_p, sv, cylct.CYL_F16, counts.numel())
        sinos.append(sv)
    del p32, counts
    prm = cylct.pose_params(0.1, 2)
    band = cylct.band(-16.0, 16.0, 12.0)
    f16 = cylct.CYL_F16
    passes = 3      # the first pass is biased on a 200 deg arc; two refinements remove it

    def one(k):
        pose, _ = cylct.cyl_estimate_pose(base, sinos[k], f16, prm)
        plan.cyl_plan_set_pose((pose[0], pose[1], 0.0, pose[3], pose[4], pose[5]))
        g, diag = plan.cyl_estimate_gamma(sinos[k], f16, xt, cylct.CYL_F32, band, passes=passes)
        return pose, g, diag

    for k in range(min(3, n_parts)):
        one(k)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    def frame(a, b, g):
        # object-to-stage rotation Rz(a) Rx(b) Rz(g) (Eq. 1)
        rz = lambda t: np.array([[math.cos(t), -math.sin(t), 0], [math.sin(t), math.cos(t), 0], [0, 0, 1]])
        rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
        return rz(a) @ rx @ rz(g)

    errs, ms, axis_err, rot_err = [], [], [], []
    for k in range(n_parts):
        t0 = time.perf_counter()
        pose, g, _ = one(k)
        ms.append((time.perf_counter() - t0) * 1e3)
        errs.append(math.degrees(math.atan2(math.sin(g - truth[k][2]), math.cos(g - truth[k][2]))))
        Oe, Ot = frame(pose[0], pose[1], g), frame(*truth[k][:3])
        axis_err.append(math.degrees(math.acos(min(1.0, float(Oe[:, 2] @ Ot[:, 2])))))
        rot_err.append(math.degrees(math.acos(max(-1.0, min(1.0, (float(np.trace(Oe.T @ Ot)) - 1.0) / 2.0)))))
    clk = clocks.stop()
    plan.close()
    e = np.abs(np.array(errs))
    t_scan = float(np.mean(ms))
    line = {
        "metric": "pose + azimuthal phase estimates per second", "value": 1e3 / t_scan, "unit": "scans/s",
        "n_gpus": 1, "steps": n_parts, "warmup": 3, "ms_per_step": t_scan, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": f"phase: {n_parts} Table 1 scans (21 views over 200 deg, 1944x1536 at 0.0748 mm, "
                               "SOD 679, SDD 791) of a tube 64 mm x R8/R3 with one off-axis pin (r 0.8 mm at "
                               "r 5.5 mm, mu 0.3), seeded pose and spin, Poisson I0 4e4, FP16; template grid "
                               "(64, 96, 32); band h in [-16, 16] mm, half-width 12 mm",
                   "step": "one scan: cyl_estimate_pose, cyl_plan_set_pose, cyl_estimate_gamma with 3 passes "
                           "(host-synchronous)"},
        "orientation_err_deg": {"mean": float(np.mean(rot_err)), "max": float(np.max(rot_err))},
        "axis_err_deg_mean": float(np.mean(axis_err)),
        "gamma_err_deg": {"mean_abs": float(e.mean()), "max_abs": float(e.max()), "rms": float(np.sqrt((e ** 2).mean())),
                          "note": "gamma alone carries the error of alpha, which a small tilt leaves poorly "
                                  "determined (Sec. 3.2); the orientation error is the rotation between the "
                                  "estimated and the true part frames"},
        "ms_per_scan": {"mean": t_scan, "median": float(np.median(ms)), "max": float(np.max(ms))},
        "clocks": clk,
        # per scan: corners, track; ray records, list (3), cuts; azimuthal mean, the mean's
        # projection and two band passes; per pass a projection, a band pass and the fit;
        # two re-poses (5 each) between and one after the passes
        "gpu_launches": (2 + 5 + 4 + 3 * 3 + 3 * 5) * n_parts,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_pose(args):
    """Pose estimation from the projections (Sec. 2.1) on Table 1's scans, as in Sec. 3.2:
    50 parts (a tube 64 mm high, 8 mm outer and 3 mm inner radius), each scanned five
    times with the stage axis on the five detector columns of Sec. 3.2; 21 projections
    over 200 deg on the 1944 x 1536 panel at 0.0748 mm, SOD 679, SDD 791; FP16 line
    integrals from Poisson counts at I0 = 4e4.  Timed: the batched estimate of all 250
    scans (one corner launch over every projection, one Levenberg-Marquardt launch), and
    one scan alone.  Precision: per part, the standard deviation of its five estimates."""
    import dataclasses
    torch, cylct = _gpu_setup()
    from paper_2005_11976_gb300 import synth
    dev = torch.device("cuda")
    n_parts = args.scans or 50
    cols = synth.TABLE1_STAGE_COLUMNS
    base = synth.table1_scan()
    # radial profile of the tube on the (1, 1, 8) grid: r in [3, 8] mm at 0.05 / mm
    rc = (np.arange(8) + 0.5) * base.radius / 8
    x = torch.from_numpy(np.where(rc >= 3.0, 0.05, 0.0).astype(np.float32).reshape(1, 1, 8)).to(dev)
    i0_pose, thr, k = 4.0e4, 0.1, 2
    rng = synth.rng_for("pose", 0)
    truth = []
    for i in range(n_parts):
        truth.append((float(rng.uniform(0, 2 * math.pi)), math.radians(float(rng.uniform(0.5, 3.0))), 0.0,
                      *[float(v) for v in rng.uniform(-2.0, 2.0, 3)]))
    scans = [dataclasses.replace(base, frames=synth.frames_from_circular(base, synth.stage_shift_mm(c)))
             for c in cols]
    sinos = []
    p32 = torch.empty(base.sino_shape, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4242)
    plans = [cylct.Plan(dataclasses.replace(sc, alpha=truth[0][0], beta=truth[0][1])) for sc in scans]
    for i in range(n_parts):
        for c, pl in enumerate(plans):
            pl.cyl_plan_set_pose(truth[i])
            pl.cyl_project(x, cylct.CYL_F32, 0, base.n_proj, p32, cylct.CYL_F32)
            counts = torch.poisson(i0_pose * torch.exp(-p32), generator=gen)
            out = torch.empty(base.sino_shape, dtype=torch.float16, device=dev)
            cylct.cyl_log_transform(counts, cylct.CYL_F32, i0_pose, out, cylct.CYL_F16, counts.numel())
            sinos.append(out)
    for pl in plans:
        pl.close()
    del p32, counts
    all_scans = [scans[c] for _ in range(n_parts) for c in range(len(cols))]
    prm = cylct.pose_params(thr, k)
    f16 = cylct.CYL_F16
    torch.cuda.synchronize()
    for _ in range(max(3, args.warmup)):
        cylct.cyl_estimate_pose_batch(all_scans, sinos, f16, prm)
    cylct.cyl_pose_set_timing(True)
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(args.steps):
        e0.record()
        poses, infos = cylct.cyl_estimate_pose_batch(all_scans, sinos, f16, prm)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    k_ms, k_n = cylct.cyl_pose_kernel_time(0)
    t_ms, t_n = cylct.cyl_pose_kernel_time(1)
    single = []
    for j in range(20):
        e0.record()
        cylct.cyl_estimate_pose(all_scans[j % len(all_scans)], sinos[j % len(sinos)], f16, prm)
        e1.record()
        e1.synchronize()
        single.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    cylct.cyl_pose_set_timing(False)
    n_scans = len(all_scans)
    t_step = float(np.mean(times))
    value = n_scans / t_step
    # precision (Sec. 3.2): std of each part's five estimates; accuracy against the truth
    P = np.array(poses).reshape(n_parts, len(cols), 6)
    T = np.array(truth)
    ax = lambda a, b: np.stack([np.sin(a) * np.sin(b), -np.cos(a) * np.sin(b), np.cos(b)], -1)
    axis_err = np.degrees(np.arccos(np.clip((ax(P[..., 0], P[..., 1]) * ax(T[:, None, 0], T[:, None, 1])).sum(-1),
                                            -1, 1)))
    prec = {"t_mm": P[..., 3:].std(axis=1).mean(axis=0).tolist(),
            "alpha_deg": float(np.degrees(P[..., 0]).std(axis=1).mean()),
            "beta_deg": float(np.degrees(P[..., 1]).std(axis=1).mean())}
    acc = {"axis_deg_mean": float(axis_err.mean()), "axis_deg_max": float(axis_err.max()),
           "t_mm_mean_abs": np.abs(P[..., 3:] - T[:, None, 3:]).mean(axis=(0, 1)).tolist()}
    # roofline of the corner pass: every pixel of every projection read once (2 bytes)
    px = base.det_w * base.det_h * base.n_proj
    bytes_launch = 2.0 * px * n_scans
    hbm, peak_kind = peaks()
    ach = bytes_launch / (k_ms / k_n / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": TRAFFIC_PER_SCAN["k_corners"] * n_scans, "kernel": "k_corners", "peak_source": peak_kind,
            "traffic_note": "ncu capture of 20 scans scaled by the scans per launch",
            "algorithmic_bytes_per_launch": bytes_launch,
            "units_per_launch": f"{n_scans} scans x 21 projections x 1944 x 1536 FP16 pixels",
            "kernel_ms_avg": {"k_corners": k_ms / k_n, "k_track_pose": t_ms / t_n},
            "kernel_share": {"k_corners": k_ms / (k_ms + t_ms), "k_track_pose": t_ms / (k_ms + t_ms)}}
    # e2e: a chunk of scans from pinned host memory through the public API
    e2e = None
    if not args.no_e2e:
        m = min(25, n_scans)
        host = [sv.cpu().pin_memory() for sv in sinos[:m]]
        dbuf = [torch.empty_like(sv) for sv in sinos[:m]]
        e0.record()
        for h, d in zip(host, dbuf):
            d.copy_(h, non_blocking=True)
        ps, _ = cylct.cyl_estimate_pose_batch(all_scans[:m], dbuf, f16, prm)
        e1.record()
        e1.synchronize()
        t_e2e = e0.elapsed_time(e1) / 1e3
        e2e = {"value": m / t_e2e, "unit": "scans/s", "h2d_bytes_per_step": int(sum(h.numel() * 2 for h in host)),
               "d2h_bytes_per_step": int(m * (6 * 8 + 72)),
               "scans_per_step": m, "note": "FP16 sinograms copied from pinned host memory, poses returned to the host"}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        from oracle import pose as opose
        oracle.build()
        s0 = dataclasses.replace(all_scans[0])
        sino0 = sinos[0].float().cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        opose.estimate_pose(oracle.Setup(**s0.fields()), sino0, thr, k)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "scans/s", "cores": 1, "kind": "oracle",
               "sample": f"one scan (21 projections of 1944 x 1536) of the workload, {dt:.2f} s"}
    line = {
        "metric": "pose estimates per second (axis detection by corner pixels + Levenberg-Marquardt)",
        "value": value, "unit": "scans/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": f"pose: Table 1 scans (21 projections over 200 deg, 1944x1536 at 0.0748 mm, "
                               f"SOD 679, SDD 791), {n_parts} parts x 5 stage positions, tube 64 mm x R8/R3, "
                               "Poisson I0 4e4, FP16 line integrals, threshold 0.1, dilation 2",
                   "l2": f"inputs {bytes_launch / 1e9:.1f} GB per step, larger than L2"},
        "baseline_note": "the paper's axis detection took 0.23 s per scan (its GPU unstated)",
        "single_scan_ms_median": float(np.median(single)),
        "precision_std_over_stage_positions": prec, "accuracy_vs_truth": acc,
        "clocks": clk, "gpu_launches": 2 * args.steps,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "batched_vs_plain": batched, "serving_vs_plain": serving,
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_compare(torch, cylct, n, rate, duration_s, part_types, ids=None):
    """Arrivals `ids` (default: all) of the first n of a Poisson stream (``rate`` scans/s) of
    the given part types through the server (continuous batching, BF16 storage, 150 GB
    budget) vs the same scans solved one at a time in arrival order.  Returns the figures
    of this process's scans (latencies per scan, in arrival order)."""
    from paper_2005_11976_gb300 import replicas, synth
    stream = [r for r in synth.serving_stream(rate, duration_s, part_types=part_types)][:n]
    if ids is not None:
        stream = [stream[i] for i in ids]
    dev = torch.device("cuda")
    bf16 = cylct.CYL_BF16
    parts = {}
    for pt in part_types:
        cfgp = synth.SERVING_PART_TYPES[pt]
        base = synth.medium_scan(n_proj=1, grid=cfgp["grid"], det=cfgp["det"], pitch=204.8 / cfgp["det"])
        rng = synth.rng_for("serving", 500 + ("small", "medium", "large").index(pt))
        az = synth.insert_azimuths(rng)
        parts[pt] = (base, synth.part_phantom(base, az), az, synth.roi_weights(base))
    t_first = stream[0][0] if ids is None or 0 in ids else synth.serving_stream(
        rate, duration_s, part_types=part_types)[0][0]      # the stream's first arrival
    # inputs of every request (projected on the GPU before the timed run)
    reqs = []
    phantoms = {}
    for k, (t_arr, pt, scan, removed) in enumerate(stream):
        base, x_warm, az, w = parts[pt]
        if (pt, removed) not in phantoms:
            phantoms[(pt, removed)] = synth.part_phantom(scan, az, removed=removed) if removed >= 0 else x_warm
        x_part = phantoms[(pt, removed)]
        with cylct.Plan(scan) as pl:
            sino = _sinogram(torch, cylct, pl, scan, x_part, I0, 200 + k, bf16)
        reqs.append((t_arr, pt, scan, sino))
    torch.cuda.synchronize()
    # ---- served
    srv = cylct.Server(150 << 30, max_active=64, n_iter=10, lam=LAMBDA, storage=bf16, weight_dtype=cylct.CYL_U8)
    pid = {}
    keep = []
    for pt, (base, x_warm, az, w) in parts.items():
        x0 = torch.from_numpy(x_warm.astype(np.float32)).to(dev).to(torch.bfloat16)
        wd = torch.from_numpy(_class_map(w)).to(dev)
        keep += [x0, wd]
        pid[pt] = srv.cyl_server_add_part(base, x0, wd)
    outs = [torch.empty(s.vol_shape, dtype=torch.bfloat16, device=dev) for _, _, s, _ in reqs]
    replicas.barrier()
    t0 = time.perf_counter()
    tickets = []
    for k, (t_arr, pt, s, sino) in enumerate(reqs):
        delay = t_arr - t_first - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.cyl_submit(pid[pt], (s.alpha, s.beta, s.gamma, s.tx, s.ty, s.tz), s.angles,
                                      sino, outs[k]))
    lat = []
    for t in tickets:
        rc, r = srv.cyl_wait(t, 3600 * 1000)
        assert rc == cylct.CYL_OK, rc
        lat.append((r.done_ns - r.submit_ns) / 1e9)
    t_served = time.perf_counter() - t0
    rounds = srv.stats()["rounds"]
    srv.close()
    # ---- plain: one cyl_sart_solve per scan, in arrival order (single-server queue)
    svc = []
    outs_p = []
    for k, (t_arr, pt, s, sino) in enumerate(reqs):
        base, x_warm, az, w = parts[pt]
        x0 = torch.from_numpy(x_warm.astype(np.float32)).to(dev).to(torch.bfloat16)
        wd = torch.from_numpy(_class_map(w)).to(dev)
        out = torch.empty(s.vol_shape, dtype=torch.bfloat16, device=dev)
        with cylct.Plan(s) as pl:
            torch.cuda.synchronize()
            a = time.perf_counter()
            pl.cyl_sart_solve(sino, bf16, x0, wd, cylct.sart_params(n_iter=10, lam=LAMBDA, weight_dtype=cylct.CYL_U8), out, bf16)
            torch.cuda.synchronize()
            svc.append(time.perf_counter() - a)
        outs_p.append(out)
    arr = [r[0] - t_first for r in reqs]
    free = 0.0
    lat_p = []
    for a, sv in zip(arr, svc):
        start = max(a, free)
        free = start + sv
        lat_p.append(free - a)
    err = max(float((outs[i].float() - outs_p[i].float()).norm() / outs_p[i].float().norm())
              for i in range(len(reqs)))
    pct = lambda v, q: float(np.percentile(np.array(v), q))
    return {"scans": len(reqs), "arrival_rate_per_s": rate, "served_scans_per_s": len(reqs) / t_served,
            "served_s": t_served, "plain_s": free, "latencies_s": lat, "plain_latencies_s": lat_p,
            "p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99),
            "plain_scans_per_s": len(reqs) / free, "plain_p50_latency_s": pct(lat_p, 50),
            "plain_p99_latency_s": pct(lat_p, 99), "served_over_plain": free / t_served,
            "max_rel_err_served_vs_plain": err, "rounds": rounds,
            "part_mix": {pt: sum(1 for r in reqs if r[1] == pt) for pt in part_types},
            "workload": f"first {len(reqs)} arrivals of a Poisson stream at {rate:g} scans/s, part types "
                        + ", ".join(f"{synth.SERVING_PART_TYPES[pt]['grid']}/{synth.SERVING_PART_TYPES[pt]['det']}^2"
                                    for pt in part_types)
                        + ", N_p in {60..360}, 10% with a removed insert, 10 sweeps, BF16 storage, 150 GB budget; "
                          "plain: the same scans one cyl_sart_solve at a time in arrival order (FIFO)"}


def run_serving(args):
    """Poisson arrivals (20 scans/s) of the three part types through the server
    (continuous batching, BF16 storage, 150 GB budget) vs the same scans solved one at a
    time in arrival order.  Under torchrun every rank serves its share of the arrivals
    (round-robin by arrival) on its own GPU; rank 0 gathers every latency."""
    torch, cylct = _gpu_setup()
    from paper_2005_11976_gb300 import replicas
    rank, world, local = replicas.dist_env()
    n = args.scans or 48
    clocks = ClockSampler(local)
    clocks.start()
    r = serving_compare(torch, cylct, n, 20.0, 600.0, ("small", "medium", "large"), replicas.shard(n, rank, world))
    clk = clocks.stop()
    dv = torch.device("cuda", local)
    t_s, t_p = replicas.max_over_ranks(r["served_s"], dv), replicas.max_over_ranks(r["plain_s"], dv)
    lat = replicas.gather_ordered(r["latencies_s"], n, rank, world)
    lat_p = replicas.gather_ordered(r["plain_latencies_s"], n, rank, world)
    err = replicas.max_over_ranks(r["max_rel_err_served_vs_plain"], dv)
    if rank == 0:
        pct = lambda v, q: float(np.percentile(np.array(v), q))
        line = {
            "metric": METRIC, "value": n / t_s, "unit": "scans/s", "n_gpus": world, "steps": 1,
            "warmup": 0, "ms_per_step": t_s * 1e3, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "serving: " + r["workload"].replace(f"first {r['scans']} ", f"first {n} "),
                       "parallelism": f"arrivals sharded over {world} GPUs" if world > 1 else "single GPU"},
            "clocks": clk, "p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99),
            "plain_scans_per_s": n / t_p, "plain_p50_latency_s": pct(lat_p, 50),
            "plain_p99_latency_s": pct(lat_p, 99), "served_over_plain": t_p / t_s,
            "max_rel_err_served_vs_plain": err,
        }
        print(json.dumps(line), flush=True)
    return 0

def _precision_oracle_cache():
    """The newest FP64 oracle result of the precision crop (written by
    ``python -m oracle.precision_reference``), read as data: (arrays, settings) or None."""
    import glob
    paths = sorted(glob.glob(os.path.join(ROOT, "oracle", "_cache", "precision_*.npz")), key=os.path.getmtime)
    if not paths:
        return None
    z = np.load(paths[-1])
    return {k: z[k] for k in z.files}, json.loads(str(z["settings"]))


def run_precision(args):
    """Precision variant (Sec. 2.2 SART with 16-bit storage): grid (256, 1024, 256), 360
    views, 512^2 detector at 0.4 mm, same phantom family as the medium workload, 30 sweeps.
    The sinogram, warm start and result are stored in FP16 or BF16; intersection math,
    accumulation and the working iterate are FP32.

    Throughput: the full workload in FP32, FP16 and BF16 storage.
    Error against the FP64 oracle, per iterate (sweeps 1, 10 and 30): on a crop of the views
    (every 90th, full grid and detector) whose oracle iterates were computed once and cached
    by ``python -m oracle.precision_reference`` (2^18 seeded voxels kept per iterate); the
    GPU solves the same crop from the same stored inputs, and the relative L2 is taken over
    the sampled voxels.
      vs_oracle_same_inputs   against the oracle fed the same stored (16-bit) inputs: the error
                              the reduced-precision path adds (bound 2e-3; FP32: 1e-5)
      vs_oracle_fp32_inputs   against the oracle fed the FP32 inputs: that error plus the
                              effect of quantising the data (information)"""
    torch, cylct = _gpu_setup()
    from paper_2005_11976_gb300 import synth
    import dataclasses
    dev = torch.device("cuda")
    F32, F16, BF16 = cylct.CYL_F32, cylct.CYL_F16, cylct.CYL_BF16
    tdt = {F32: torch.float32, F16: torch.float16, BF16: torch.bfloat16}
    names = {F32: "f32", F16: "f16", BF16: "bf16"}
    kmax = 30
    # the same draws as the cached oracle run: the pose from one generator, the inserts from
    # a fresh one
    scan = synth.precision_scan(synth.rng_for("precision"))
    rng = synth.rng_for("precision")
    az = synth.insert_azimuths(rng)
    removed = int(rng.integers(8))
    x_warm = synth.part_phantom(scan, az)
    x_part = synth.part_phantom(scan, az, removed=removed)
    w = synth.roi_weights(scan)
    wd = torch.from_numpy(_class_map(w)).to(dev)
    x0_32 = torch.from_numpy(x_warm.astype(np.float32)).to(dev)

    def solve(plan, sino, x0, dt, k):
        out = torch.empty(plan.scan.vol_shape, dtype=tdt[dt], device=dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.cyl_sart_solve(sino, dt, x0, wd, cylct.sart_params(n_iter=k, lam=LAMBDA, weight_dtype=cylct.CYL_U8),
                            out, dt)
        e1.record()
        e1.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    clocks = ClockSampler(0)
    clocks.start()
    # ---- throughput of the full workload
    plan = cylct.Plan(scan)
    sino32 = _sinogram(torch, cylct, plan, scan, x_part, I0, 300, F32)
    rates = {}
    for dt in (F32, F16, BF16):
        out, t = solve(plan, sino32.to(tdt[dt]), x0_32.to(tdt[dt]), dt, kmax)
        rates[names[dt]] = kmax / t
        del out
    # kernel times of one FP32 sweep (a CUDA event between launches): a grid twice the L2
    plan.cyl_plan_set_timing(True)
    solve(plan, sino32, x0_32, F32, 1)
    plan.cyl_plan_set_timing(False)
    k_ms, k_n = zip(*[plan.cyl_plan_kernel_time(k) for k in range(3)])
    cnt = torch.empty(scan.n_proj, dtype=torch.int64, device=dev)
    plan.cyl_count_segments(0, scan.n_proj, cnt)
    S = float(cnt.float().mean().item())
    n_pix, n_vox = scan.det_w * scan.det_h, scan.n_vox
    avg = {"k_sart": k_ms[0] / max(k_n[0], 1) / 1e3, "k_update_nd4": k_ms[2] / max(k_n[2], 1) / 1e3}
    hbm, peak_kind = peaks()
    fwd, back, upd = S * 4 + n_pix * 8, S * 4, 2 * n_vox * 4 + n_vox
    roof = {"bound": "hbm", "peak": hbm, "peak_source": peak_kind, "unit": "GB/s", "segments_per_view": S,
            "model": "segment-touch (path specification), FP32",
            "kernel_us_avg": {k: v * 1e6 for k, v in avg.items()},
            "kernel_frac": {"k_sart": (fwd + back) / avg["k_sart"] / 1e9 / hbm,
                            "k_update_nd4": upd / avg["k_update_nd4"] / 1e9 / hbm},
            "path_per_view_frac": (fwd + back + upd) / (avg["k_sart"] + avg["k_update_nd4"]) / 1e9 / hbm}
    plan.close()
    del sino32
    # ---- per-iterate error against the oracle on the cached crop
    errors = None
    cache = _precision_oracle_cache()
    if cache is not None:
        z, st = cache
        crop = dataclasses.replace(scan, angles=scan.angles[::st["view_step"]])
        assert np.allclose(crop.angles, st["scan"]["angles"]) and crop.n_vox == st["scan"]["n_h"] * \
            st["scan"]["n_theta"] * st["scan"]["n_r"], "the cached crop is not this workload's"
        idx = torch.from_numpy(z["idx"]).to(dev)
        p32 = torch.from_numpy(z["p_f32"].reshape(crop.sino_shape)).to(dev)
        errors = {"crop": f"views 0::{st['view_step']} ({crop.n_proj}) of the precision workload, full grid and "
                          f"detector; {len(z['idx'])} sampled voxels", "vs_oracle_same_inputs": {},
                  "vs_oracle_fp32_inputs": {}}
        with cylct.Plan(crop) as cp:
            for dt in (F32, F16, BF16):
                nm = names[dt]
                same, f32in = {}, {}
                for k in st["sweeps"]:
                    out, _ = solve(cp, p32.to(tdt[dt]), x0_32.to(tdt[dt]), dt, k)
                    g = out.float().reshape(-1)[idx].double().cpu().numpy()
                    ref = z[f"{nm}_sweep{k}"]
                    ref32 = z[f"f32_sweep{k}"]
                    same[k] = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
                    f32in[k] = float(np.linalg.norm(g - ref32) / np.linalg.norm(ref32))
                errors["vs_oracle_same_inputs"][nm] = same
                if dt != F32:
                    errors["vs_oracle_fp32_inputs"][nm] = f32in
    clk = clocks.stop()
    line = {
        "metric": METRIC, "value": rates["bf16"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": kmax / rates["bf16"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "precision: grid (256,1024,256) R25 H50, 360 views, 512x512 det 0.4 mm, "
                               f"{kmax} sweeps lambda 0.5, warm start, ROI weights (U8 class map), Poisson I0 1e4; "
                               "sinogram, warm start and result stored in FP16 / BF16, FP32 math and iterate"},
        "sart_iters_per_s": rates,
        "rel_l2_per_iterate": errors if errors is not None else "no cached oracle result: run python -m oracle.precision_reference",
        "bound": "vs_oracle_same_inputs <= 2e-3 (16-bit storage), <= 1e-5 (FP32)",
        "roofline_fp32_sweep": roof,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


# The path's memory work is scattered single-sector gathers and reductions, not streams:
# this probe measures the GPU's rate for exactly those, at the medium view's sizes, so
# that the kernels can be set against it.  Every index is reduced modulo the buffer length.
L2OPS_SRC = r"""
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("ERR %s\n", cudaGetErrorString(e)); return 1; } } while (0)
__device__ __forceinline__ uint32_t mix(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16; return x;
}
__device__ __forceinline__ void red2(float2 *p, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" :: "l"(p), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void red4(float2 *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" :: "l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}
// 0: 8-byte reductions at random voxels; 1: 16-byte reductions at random voxel pairs;
// 2: 8-byte reductions along random walks (steps +-1, +-N_r, +N_theta N_r, like a ray);
// 3: 4-byte gathers at random voxels; 4: 4-byte gathers along random walks
__global__ void k(int mode, float2 *nd, const float *x, uint32_t n, int per, float *sink, int nr, int ntnr) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    uint32_t h = mix(tid * 2654435761u + 12345u), idx = h % n;
    for (int i = 0; i < per; ++i) {
        h = mix(h + i);
        if (mode == 0) red2(nd + (h % n), 1.f, 0.5f);
        else if (mode == 1) red4(nd + ((h % n) & ~1u), 1.f, 0.5f, 1.f, 0.5f);
        else if (mode == 3) acc += __ldg(x + (h % n));
        else {
            const uint32_t r = h & 7;
            const int d = r < 4 ? ((r & 1) ? 1 : -1) : (r < 7 ? ((r & 1) ? nr : -nr) : ntnr);
            idx = (uint32_t)(((int64_t)idx + d + n) % n);
            if (mode == 2) red2(nd + idx, 1.f, 0.5f); else acc += __ldg(x + idx);
        }
    }
    if (acc == 123.456f) sink[0] = acc;
}
int main() {
    const uint32_t n = 128u * 512u * 128u;
    float2 *nd; float *x, *sink;
    CK(cudaMalloc(&nd, sizeof(float2) * n)); CK(cudaMalloc(&x, sizeof(float) * n)); CK(cudaMalloc(&sink, 64));
    CK(cudaMemset(nd, 0, sizeof(float2) * n)); CK(cudaMemset(x, 0, sizeof(float) * n));
    int nsm; CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0));
    cudaEvent_t a, b; CK(cudaEventCreate(&a)); CK(cudaEventCreate(&b));
    const double ops_total = 18.45e6;
    for (int mode = 0; mode < 5; ++mode)
        for (int bps = 2; bps <= 8; bps *= 2) {
            const int threads = 256, blocks = nsm * bps;
            const int per = (int)(ops_total / ((double)threads * blocks) + 0.5);
            for (int r = 0; r < 2; ++r) k<<<blocks, threads>>>(mode, nd, x, n, per, sink, 128, 512 * 128);
            CK(cudaEventRecord(a));
            for (int r = 0; r < 5; ++r) k<<<blocks, threads>>>(mode, nd, x, n, per, sink, 128, 512 * 128);
            CK(cudaEventRecord(b)); CK(cudaEventSynchronize(b));
            float ms; CK(cudaEventElapsedTime(&ms, a, b));
            printf("%d %d %.6e\n", mode, bps, (double)per * threads * blocks * 5 / (ms * 1e-3));
        }
    CK(cudaDeviceSynchronize());
    return 0;
}
"""


def run_l2ops(args):
    """Rates of scattered L2 work on this GPU: reductions and gathers of the medium view's
    sizes (8.39 M voxels), random and along ray-like walks, at 2, 4 and 8 blocks per SM."""
    import tempfile
    from paper_2005_11976_gb300 import build as cbuild
    names = {0: "red.v2 random", 1: "red.v4 random (voxel pairs)", 2: "red.v2 walk",
             3: "gather 4 B random", 4: "gather 4 B walk"}
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l2ops.cu"), os.path.join(d, "l2ops")
        with open(src, "w") as f:
            f.write(L2OPS_SRC)
        subprocess.run([cbuild.nvcc()] + cbuild.ARCH + ["-O3", "-o", exe, src], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    rates = {}
    for ln in out.split("\n"):
        parts = ln.split()
        if len(parts) == 3:
            rates.setdefault(names[int(parts[0])], {})[f"{parts[1]}_blocks_per_sm"] = float(parts[2]) / 1e9
    best = {k: max(v.values()) for k, v in rates.items()}
    line = {"metric": "scattered L2 operations per second", "value": best["red.v2 random"], "unit": "G ops/s",
            "n_gpus": 1, "steps": 5, "warmup": 2, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "l2ops: 18.45 M operations per launch over 8.39 M voxels (float2 accumulator, "
                                   "float volume), 256-thread blocks"},
            "g_ops_per_s": rates, "best_g_ops_per_s": best}
    print(json.dumps(line), flush=True)
    return 0


def run_mtf(args):
    """Directional MTF (Sec. 2.3, Eq. 8) of SART on the cylindrical grid: azimuthal
    (Siemens-star) and radial (concentric-circle) cosine line phantoms with n_l = 1 .. 128
    lines, simulated on a fine (32, 1608, 256) grid, projected (360 views over 360 deg,
    1024 x 128 detector at 0.2 mm), reconstructed on (32, 512, 256) by 5 sweeps of SART from
    zero with the non-negativity clamp; the modulation of the central slice per radius.  Then the few-view study of
    Sec. 3.1: 67 views, reconstructed with N_theta = 512 and with N_theta = 64."""
    torch, cylct = _gpu_setup()
    from paper_2005_11976_gb300 import mtf, synth
    dev = torch.device("cuda")
    n_views = args.scans or 360
    sweeps = 5
    R, H = 25.0, 6.4

    def scan(grid, n_proj):
        return synth.Scan(*grid, R, H, 200.0, 800.0, 1024, 128, 0.2, 0.2, synth.full_circle(n_proj))

    fine, rec_shape = (32, 1608, 256), (32, 512, 256)
    results = {"theta": {}, "r": {}}
    few = {"theta": {}, "r": {}}
    t_sim = t_rec = t_main = 0.0
    n_main = 0
    clocks = ClockSampler(0)
    clocks.start()
    with cylct.Plan(scan(fine, n_views)) as sim, cylct.Plan(scan(rec_shape, n_views)) as rec, \
            cylct.Plan(scan(fine, 67)) as sim67, cylct.Plan(scan(rec_shape, 67)) as rec67, \
            cylct.Plan(scan((32, 64, 256), 67)) as rec67_64:
        def run(sim_plan, rec_plan, kind, n_l, n_p, shape):
            nonlocal t_sim, t_rec, t_main, n_main
            x = torch.from_numpy(mtf.line_phantom(kind, n_l, fine).astype(np.float32)).to(dev)
            p = torch.empty((n_p, 128, 1024), device=dev)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            out = torch.empty(shape, device=dev)
            e0.record()
            sim_plan.cyl_project(x, cylct.CYL_F32, 0, n_p, p, cylct.CYL_F32)
            e1.record()
            # attenuation is non-negative: Eq. 8 lies in [0, 1] for positive mu
            rec_plan.cyl_sart_solve(p, cylct.CYL_F32, None, None,
                                    cylct.sart_params(n_iter=sweeps, lam=LAMBDA, clamp_nonneg=True),
                                    out, cylct.CYL_F32)
            e2.record()
            e2.synchronize()
            t_sim += e0.elapsed_time(e1) / 1e3
            t_rec += e1.elapsed_time(e2) / 1e3
            if n_p == n_views:
                t_main += e1.elapsed_time(e2) / 1e3
                n_main += sweeps
            return out.cpu().numpy().astype(np.float64)

        for kind in ("theta", "r"):
            for n_l in mtf.frequencies(256):
                x = run(sim, rec, kind, n_l, n_views, rec_shape)
                if kind == "theta":
                    radii = (np.arange(rec_shape[2]) + 0.5) / rec_shape[2]
                    m = mtf.mtf_theta(x)
                else:
                    radii, m = mtf.mtf_r(x, n_l)
                results[kind][n_l] = {"mean": float(m.mean()), "by_radius": mtf.summarise(m, radii)}
                row = {}
                for label, plan67, shape in (("n_theta_512", rec67, rec_shape), ("n_theta_64", rec67_64, (32, 64, 256))):
                    x67 = run(sim67, plan67, kind, n_l, 67, shape)
                    if kind == "theta":
                        r67 = (np.arange(shape[2]) + 0.5) / shape[2]
                        m67 = mtf.mtf_theta(x67)
                    else:
                        r67, m67 = mtf.mtf_r(x67, n_l)
                    row[label] = {"mean": float(m67.mean()), "by_radius": mtf.summarise(m67, r67)}
                few[kind][n_l] = row
    clk = clocks.stop()
    line = {
        "metric": METRIC, "value": n_main / t_main if t_main else None,
        "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": (t_sim + t_rec) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"MTF: cosine line phantoms n_l = 1..128 on a (32,1608,256) grid, {n_views} views "
                               "1024x128 at 0.2 mm, SOD 200 SDD 800, R 25 H 6.4; SART 5 sweeps from zero on "
                               "(32,512,256), non-negativity clamp; 67-view study with N_theta 512 and 64"},
        "mtf_theta": results["theta"], "mtf_r": results["r"],
        "few_views_67": few,
        "seconds": {"simulation": t_sim, "reconstruction": t_rec},
        "value_is": f"SART sweeps/s of the {n_views}-view (32,512,256) reconstructions",
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
