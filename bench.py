"""Benchmark: FBS iterations/s of the full multigrid reconstruction on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload medium]
    python -m torch.distributed.run --nproc-per-node N ... bench.py --gpus N

A step is one complete ``cbct_reconstruct`` call (Algorithm A1 on every multigrid
level: forward projection + residual, adjoint gather + gradient step, M TV-prox
sweeps with f >= 0, float64 energies; the automatic beta's power iterations; the
2x2 data binning and the prolongations) on seeded synthetic data of the workload's
shape.  Inputs are resident in HBM when the timed region starts; L2 is flushed
(256 MiB write) between steps, outside the timed events.  Each GPU runs independent
reconstructions (no data-path collective; weak scaling).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead, on
the host cores, one Algorithm A1 iteration of the finest level per step.

Two serving modes print their own line (reconstructions/s):

* ``--mode batch``: 16 heterogeneous requests (six volume sizes from 128^3 to
  384x384x64, 20-60 views, random start angles, 2 levels x 30 iterations), run one at
  a time through ``cbct_reconstruct`` and together through ``cbct_reconstruct_batch``;
  ``--batch-mix small --requests 32`` takes 32 requests of the small workload instead.
* ``--mode serve``: requests (by default drawn uniformly from the medium workload and
  the large one at 20, 30 and 40 views; ``--mix batch16`` takes the 16 requests above)
  arrive as a Poisson stream at a fixed fraction of the one-at-a-time capacity and go
  through the continuous-batching server with a 150 GB budget; latency percentiles are
  compared with a one-at-a-time FIFO queue fed the same arrival times and the
  measured per-request service times.
* ``--mode vcycle``: V-cycles (mg_cycle 1) against the cascade on the workload: time
  per reconstruction and the energy of Eq. 1 each reaches.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD_TEXT = {
    "small": "64^3 @ 4 mm, 20 views 64x48 @ 8 mm, noise-free, 1 level x 20 FBS iterations",
    "medium": "256x256x64 @ 1x1x2.5 mm, 40 views 256x192 @ 1.6 mm, Poisson I0=1e5, 2-level multigrid "
              "x 50 FBS iterations per level",
    "large": "512x512x96 @ 0.5x0.5x2.5 mm, 40 views 512x384 @ 0.8 mm, Poisson I0=2.5e4, 3-level multigrid "
             "x 50 FBS iterations per level",
    "large30": "512x512x96 @ 0.5x0.5x2.5 mm, 30 views 512x384 @ 0.8 mm, Poisson I0=2.5e4, 3-level multigrid "
               "x 50 FBS iterations per level",
    "large20": "512x512x96 @ 0.5x0.5x2.5 mm, 20 views 512x384 @ 0.8 mm, Poisson I0=2.5e4, 3-level multigrid "
               "x 50 FBS iterations per level",
}
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
# Lane-operations per nonzero that no implementation of the exact-length operators can
# avoid: adjoint 8 (two z-crossings: 2 sub + 2 mul, clip:
# 1 max + 1 min, length: 1 sub, accumulate: 1 fma); projector 4 (pick next crossing:
# 1 min, length: 1 sub, accumulate: 1 fma, advance the crossing: 1 fma).
OPS_PER_NNZ = {"backproject": 8.0, "project": 4.0}
# Sources of each timed kernel; the DRAM traffic recorded in profiles/ counts only while
# they are unchanged since the capture.
KERNEL_SOURCES = {
    "backproject": ("k_backproject", ["k_backproject.cu", "bp_tile.cuh"]),
    "project": ("k_project", ["k_project.cu", "project_tile.cuh"]),
    "tv": ("k_tv_sweep", ["k_tv.cu", "tv_tile.cuh"]),
}


def profile_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, or None when there is no
    summary for this workload or the kernel's sources changed since it was taken."""
    import hashlib
    import re
    name, files = KERNEL_SOURCES[kernel]
    try:
        text = open(os.path.join(ROOT, "profiles", f"{name}_{workload}.md")).read()
        h = hashlib.sha256()
        for f in files:
            with open(os.path.join(ROOT, "paper_1002_3675_b300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    t = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    s = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    if not t or not s or s.group(1) != h.hexdigest()[:16]:
        return None
    return int(t.group(1))


def load_nnz(workload):
    with open(os.path.join(ROOT, "tests", "golden", "nnz.json")) as fh:
        return [lv["nnz"] for lv in json.load(fh)[workload]]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu_index):
        self.p = None
        self.path = os.path.join(os.environ.get("CBCT_CLOCK_LOG_DIR", tempfile.gettempdir()),
                                 f"clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={CLOCK_QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_oracle_iterations(case, n_iter):
    """Time n_iter Algorithm A1 iterations of the oracle on the finest level."""
    import oracle
    g = case["geom"]
    mu = case["mu"]
    eps = oracle.default_eps(g)
    beta = 1.05 * oracle.gamma(g, mu) * 1.6e4  # fixed value of the right size; not timed work
    Y = np.asarray(case["Y"], dtype=np.float64)
    f0 = np.zeros((g["nz"], g["ny"], g["nx"]))
    t0 = time.perf_counter()
    oracle.fbs(g, Y, mu, beta, eps, 10, n_iter, f0=f0)
    return time.perf_counter() - t0, oracle.num_threads()


def run_reference(args, world, rank):
    if rank != 0:
        return
    case = synth.make_case(args.workload)
    for _ in range(args.warmup):
        cpu_oracle_iterations(case, 1)
    times = []
    for _ in range(args.steps):
        dt, cores = cpu_oracle_iterations(case, 1)
        times.append(dt)
    tot = sum(times)
    value = args.steps / tot
    sample = (f"1 Algorithm A1 iteration (P, P^T, 10 prox sweeps) of the finest level per step "
              f"({WORKLOAD_TEXT[args.workload].split(',')[0]}), {args.steps} steps")
    line = {"impl": "reference", "metric": "FBS iterations/s", "value": value, "unit": "iter/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded ellipsoid phantom, analytic line integrals, Poisson/log noise)",
            "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}", "host_cores": os.cpu_count(),
                       "note": "the FP64 oracle on the host cores (rank 0 only); n_gpus is the launch's rank count"},
            "cpu_baseline": {"value": value, "unit": "iter/s", "cores": cores, "cpu_model": cpu_model(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, world, rank, local):
    import torch

    from paper_1002_3675_b300 import cbct

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = synth.CONFIGS[args.workload]
    case = synth.make_case(args.workload)
    G = cbct.cbct_geometry_create(case["geom"])
    levels, iters, mu = cfg["levels"], cfg["iters"], cfg["mu"]
    Y_host = torch.tensor(np.asarray(case["Y"], dtype=np.float32)).pin_memory()
    Y = Y_host.to(dev)
    f = torch.empty((cfg["vol"][2], cfg["vol"][1], cfg["vol"][0]), dtype=torch.float32, device=dev)
    f_host = torch.empty(f.shape, dtype=torch.float32).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # the timed steps time the two operator classes launch by launch (CUDA events on the
    # launching stream); every class is timed in a separate pass after the timed region
    timed_mask = (1 << cbct.KERNEL_CLASSES.index("project")) | (1 << cbct.KERNEL_CLASSES.index("backproject"))

    def step(kernel_times, mask=timed_mask, serial_power=False):
        return cbct.cbct_reconstruct(G, Y, mu, iters, levels, f_out=f, kernel_times=kernel_times, kernel_mask=mask,
                                     tv_mode=args.tv_mode, adjoint_mode=args.adjoint_mode, sino_fp16=args.sino_fp16,
                                     serial_power=serial_power)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()

    # ---- device-resident timed region --------------------------------------------
    sampler = ClockSampler(local) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    step_ms, kms, klaunch, kms_f, kl_f = [], {}, {}, {}, {}
    n_launch0 = cbct.cbct_kernel_launch_count()
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = step(True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for k, v in info["kernel_ms"].items():
            kms[k] = kms.get(k, 0.0) + v
        for k, v in info["kernel_launches"].items():
            klaunch[k] = klaunch.get(k, 0) + v
        for k, v in info["kernel_ms_finest"].items():
            kms_f[k] = kms_f.get(k, 0.0) + v
        for k, v in info["kernel_launches_finest"].items():
            kl_f[k] = kl_f.get(k, 0) + v
    torch.cuda.synchronize()
    n_launch = cbct.cbct_kernel_launch_count() - n_launch0
    barrier(world)
    clocks = sampler.stop() if sampler else None
    tot_ms = max_over_ranks(sum(step_ms), world)
    n_iter = levels * iters
    value = world * args.steps * n_iter / (tot_ms / 1e3)

    # ---- end to end through the C ABI with host buffers ---------------------------
    barrier(world)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Y.copy_(Y_host, non_blocking=True)
        step(False)
        f_host.copy_(f, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_tot = max_over_ranks(sum(e2e_ms), world)
    e2e_value = world * args.steps * n_iter / (e2e_tot / 1e3)

    # ---- every kernel class timed launch by launch (a separate pass of the same steps, the
    #      power iterations in level order so that no two streams share the event windows) --
    split_ms, split_n = {}, {}
    for _ in range(args.steps):
        flush.fill_(1)
        _, info = step(True, mask=0, serial_power=True)
        for k, v in info["kernel_ms"].items():
            split_ms[k] = split_ms.get(k, 0.0) + v
        for k, v in info["kernel_launches"].items():
            split_n[k] = split_n.get(k, 0) + v
    torch.cuda.synchronize()

    # ---- the same steps with lambda_max(P^T P) cached per geometry (reported beside) --
    cbct.cbct_reconstruct(G, Y, mu, iters, levels, f_out=f, reuse_lambda=True, tv_mode=args.tv_mode,
                          adjoint_mode=args.adjoint_mode, sino_fp16=args.sino_fp16)   # fills the cache
    torch.cuda.synchronize()
    cached_ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cbct.cbct_reconstruct(G, Y, mu, iters, levels, f_out=f, reuse_lambda=True, tv_mode=args.tv_mode,
                              adjoint_mode=args.adjoint_mode, sino_fp16=args.sino_fp16)
        e1.record(stream)
        e1.synchronize()
        cached_ms.append(e0.elapsed_time(e1))
    cached_tot = max_over_ranks(sum(cached_ms), world)

    if rank != 0:
        return

    # ---- roofline of the dominant kernel --------------------------------------------
    peaks, peak_kind = measured_peaks()
    nnz = load_nnz(args.workload)
    K_pi = 30
    units = {  # nonzeros processed per reconstruction by each operator
        "project": sum(n * (iters + K_pi) for n in nnz),
        "backproject": sum(n * (iters + K_pi) for n in nnz),
    }
    # the Eq. 2 adjoint variant mixes two adjoints in one class: no nonzero-based rate
    candidates = ("project", "backproject", "tv") if args.adjoint_mode == 0 else ("project", "tv")
    dom = max(candidates, key=lambda k: split_ms.get(k, 0.0))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_mhz = (clocks or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") \
        or peaks.get("sm_max_mhz", 2032.0)
    alu_peak = sm_count * 128 * clock_mhz * 1e6 / 1e12      # T lane-ops/s (FP32 pipes x clock)
    # rates from the finest level's Algorithm A1 iterations, timed inside the timed steps:
    # they run after every power iteration has finished, so nothing shares their event
    # windows (the finer levels' power iterations overlap the coarser levels on a side
    # stream); the per-class totals come from the separate serial pass
    units_f = {k: nnz[0] * iters for k in ("project", "backproject")}
    per_kernel = {}
    for k in ("project", "backproject"):
        t = kms_f[k] / 1e3
        per_kernel[k] = {"ms_per_step": split_ms[k] / args.steps, "launches_per_step": split_n[k] / args.steps,
                         "finest_fbs_ms_per_step": kms_f[k] / args.steps,
                         "finest_fbs_launches_per_step": kl_f[k] / args.steps}
        if k == "backproject" and args.adjoint_mode == 1:
            per_kernel[k]["note"] = "Eq. 2 adjoint in the FBS iterations: no nonzero-based rate"
            continue
        per_kernel[k]["gnnz_per_s"] = units_f[k] * args.steps / t / 1e9
        per_kernel[k]["alu_tops"] = units_f[k] * args.steps * OPS_PER_NNZ[k] / t / 1e12
    nvox = [np.prod([(n + (1 << l) - 1) >> l for n in cfg["vol"]]) for l in range(levels)]
    tv_bytes = sum(12.0 * v * iters * 10 for v in nvox) * args.steps   # read f, read g, write f per sweep
    per_kernel["tv"] = {"ms_per_step": split_ms["tv"] / args.steps,
                        "gbs": tv_bytes / (split_ms["tv"] / 1e3) / 1e9, "launches_per_step": split_n["tv"] / args.steps,
                        "note": "timed in the separate all-classes pass"}
    if dom in ("project", "backproject"):
        ach = per_kernel[dom]["alu_tops"]
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "Tlane-op/s",
                "frac": ach / alu_peak, "traffic": profile_traffic(dom, args.workload),
                "launch_ms": kms_f[dom] / (args.steps * iters),
                "timing": "CUDA events around every operation of the class in the finest level's Algorithm A1 "
                          "iterations inside the timed steps (no other stream's work beside them); launch_ms is "
                          "the time of one operation (the adjoint: column running sums + gather)",
                "basis": f"{OPS_PER_NNZ[dom]:.0f} lane-ops per nonzero x the finest level's exact nnz; peak = "
                         f"{sm_count} SMs x 128 FP32 lanes x {clock_mhz:.0f} MHz (median SM clock in the timed "
                         "region)"}
    else:
        ach = per_kernel["tv"]["gbs"]
        roof = {"kernel": "tv", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": profile_traffic("tv", args.workload)}
    roof["peak_source"] = peak_kind

    # ---- CPU baseline: the oracle on a bounded sample ---------------------------------
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        n_cpu = 2
        dt, cores = cpu_oracle_iterations(case, n_cpu)
        cpu = {"value": n_cpu / dt, "unit": "iter/s", "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"{n_cpu} Algorithm A1 iterations (P, P^T, 10 prox sweeps) of the finest level of the "
                         f"same workload, FP64 C oracle with OpenMP; fixed beta, no power iteration"}

    # ---- per-iteration fractions (algorithmic HBM bytes and the composite floor) -------
    s_bytes = 2 if args.sino_fp16 else 4
    dims = [cbct.cbct_level_dims(G, l) for l in range(levels)]
    nv_l = [d[0] * d[1] * d[2] for d in dims]
    nr_l = [len(case["geom"]["angles"]) * d[3] * d[4] for d in dims]
    b_fbs = sum(24 * v + (8 + s_bytes) * r for v, r in zip(nv_l, nr_l)) * iters       # per step
    b_pow = sum(8 * v + 8 * r for v, r in zip(nv_l, nr_l)) * K_pi
    bw = peaks["hbm_gbs"] * 1e9
    t_step = tot_ms / args.steps / 1e3
    floor_s = {"project": units["project"] * OPS_PER_NNZ["project"] / (alu_peak * 1e12),
               "backproject": units["backproject"] * OPS_PER_NNZ["backproject"] / (alu_peak * 1e12),
               "tv": sum(12.0 * v * 10 for v in nv_l) * iters / bw}
    per_iter = {"hbm_bytes_per_fbs_iteration_finest": 24 * nv_l[0] + (8 + s_bytes) * nr_l[0],
                "literal_hbm_frac": (b_fbs + b_pow) / (t_step * bw),
                "composite_frac": sum(floor_s.values()) / t_step,
                "floor_ms_per_step": {k: v * 1e3 for k, v in floor_s.items()},
                "basis": "literal: (24 Nv + (8+s) Nr) bytes per FBS iteration and (8 Nv + 8 Nr) per power "
                         "iteration over the step time at the measured HBM bandwidth; composite: the sum of "
                         "the per-class floors (P and P^T: nonzeros x lane-ops / FP32 issue peak; TV: 12 B "
                         "per voxel per sweep / HBM) over the step time"}

    # ---- quality context: the last reconstruction against the ground truth ------------
    quality = None
    if not args.no_quality:
        gm = case["geom"]
        ss = 1 if gm["nx"] * gm["ny"] * gm["nz"] > 8e6 else 2
        truth = synth.voxelize(case["ellipsoids"], gm, ss)
        rec = f.detach().cpu().numpy().astype(np.float64)
        z = (np.arange(gm["nz"]) - (gm["nz"] - 1) / 2) * gm["hz"]
        y = (np.arange(gm["ny"]) - (gm["ny"] - 1) / 2) * gm["hy"]
        x = (np.arange(gm["nx"]) - (gm["nx"] - 1) / 2) * gm["hx"]
        r_xy = np.sqrt(y[:, None] ** 2 + x[None, :] ** 2)
        r_fov = gm["dso"] * np.sin(np.arctan(gm["nu"] * gm["du"] / 2 / gm["dsd"]))
        z_cov = gm["nv"] * gm["dv"] / 2 * (gm["dso"] - r_xy) / gm["dsd"]
        mask = (r_xy[None] <= r_fov) & (np.abs(z)[:, None, None] <= z_cov[None])
        eps_d = 2e-5 / min(gm["hx"], gm["hy"], gm["hz"])
        E = cbct.cbct_energy(G, Y, f, mu, eps_d, tv_mode=args.tv_mode)
        E0 = cbct.cbct_energy(G, Y, f, mu, 0.0, tv_mode=args.tv_mode)
        quality = {"rmse_fully_sampled": float(np.sqrt(np.mean((rec - truth)[mask] ** 2))),
                   "truth_rms_fully_sampled": float(np.sqrt(np.mean(truth[mask] ** 2))),
                   "fully_sampled_fraction": float(mask.mean()), "unit": "1/mm",
                   "E": float(E[0]), "E1_eps": float(E[1]), "E1_exact": float(E0[1]), "muE2": float(E[2]),
                   "truth": f"ellipsoid phantom voxelised with {ss}^3 sub-samples per voxel",
                   "region": "inside the transverse field of view and the cone seen from every view"}

    # ---- float16 data storage: the reconstruction against the float32 one ------------
    fp16_err = None
    if args.sino_fp16:
        f32r = torch.empty_like(f)
        cbct.cbct_reconstruct(G, Y, mu, iters, levels, f_out=f32r, tv_mode=args.tv_mode,
                              adjoint_mode=args.adjoint_mode)
        a64, b64 = f.double(), f32r.double()
        fp16_err = {"rel_l2_vs_float32_data": float(torch.linalg.vector_norm(a64 - b64) /
                                                    torch.linalg.vector_norm(b64)),
                    "note": "the same reconstruction with float32 data storage (within 1e-4 of the FP64 "
                            "oracle by the parity tests)"}

    launches = int(n_launch)   # every kernel the library launched inside the timed region
    line = {
        "metric": "FBS iterations/s", "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ellipsoid phantom, analytic line integrals, Poisson/log noise); "
                "stands in for the paper's NCAT/CatPhan data",
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}", "inner_iters": 10,
                   "variant": {"tv_mode": ["isotropic", "anisotropic"][args.tv_mode],
                               "adjoint": ["exact transpose", "Eq. 2 interpolation"][args.adjoint_mode],
                               "data_storage": "float16" if args.sino_fp16 else "float32"},
                   "beta": "auto per level (30 power iterations, recomputed every step)",
                   "fbs_iterations_per_step": n_iter, "l2": "flushed between steps (256 MiB write, untimed)",
                   "parallelism": f"replicas x{world}"},
        "recon_s": tot_ms / args.steps / 1e3,
        "e2e": {"value": e2e_value, "unit": "iter/s", "h2d_bytes_per_step": int(Y_host.numel() * 4),
                "d2h_bytes_per_step": int(f_host.numel() * 4)},
        "lambda_cached": {"value": world * args.steps * n_iter / (cached_tot / 1e3), "unit": "iter/s",
                          "ms_per_step": cached_tot / args.steps,
                          "note": "beta's power iterations reused from an earlier call on the same geometry"},
        "roofline": roof,
        "kernels": per_kernel,
        "kernel_ms_per_step": {k: v / args.steps for k, v in split_ms.items()},
        "kernel_split_note": "kernel_ms_per_step: every launch timed with CUDA events in a separate pass of the "
                             "same steps, the power iterations in level order (serial_power); the timed steps "
                             "time the project and backproject launches, and the rates and the roofline use "
                             "those of the finest level's Algorithm A1 iterations",
        "gpu_launches": launches,
        "per_iteration": per_iter,
        "quality": quality,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if fp16_err is not None:
        line["fp16_error"] = fp16_err
    print(json.dumps(line), flush=True)


def _upload_requests(reqs, dev):
    import torch
    out = []
    for r in reqs:
        g = r["geom"]
        out.append(dict(r, Y_dev=torch.tensor(np.asarray(r["Y"], dtype=np.float32), device=dev),
                        f_dev=torch.zeros((g["nz"], g["ny"], g["nx"]), dtype=torch.float32, device=dev)))
    return out


def _request_text(reqs):
    sizes = sorted({(r["geom"]["nx"], r["geom"]["ny"], r["geom"]["nz"]) for r in reqs})
    views = [len(r["geom"]["angles"]) for r in reqs]
    return (f"{len(reqs)} requests, volumes {', '.join('x'.join(map(str, s)) for s in sizes)}, "
            f"{min(views)}-{max(views)} views, {reqs[0]['levels']} levels x {reqs[0]['iters']} FBS iterations, "
            f"Poisson I0 1e4-1e5")


def _sequential(cbct, reqs, stream):
    """Per-request service times (s) of one-at-a-time cbct_reconstruct calls."""
    import torch
    times = []
    for r in reqs:
        G = r["G"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cbct.cbct_reconstruct(G, r["Y_dev"], r["mu"], r["iters"], r["levels"], f_out=r["f_dev"])
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return times


def _small_requests(n, seed):
    """n requests of the small workload (64^3, 20 views) with random start angles."""
    rng = np.random.default_rng(seed)
    cfg = synth.CONFIGS["small"]
    out = []
    for _ in range(n):
        c = synth.make_case("small", theta0=float(rng.uniform(0.0, 2.0 * np.pi / cfg["n_angles"])))
        out.append(dict(geom=c["geom"], Y=c["Y"], mu=cfg["mu"], levels=cfg["levels"], iters=cfg["iters"]))
    return out


def run_batch(args, world, rank, local):
    import torch

    from paper_1002_3675_b300 import cbct

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.batch_mix == "small":
        reqs = _upload_requests(_small_requests(args.requests, 1005 + rank), dev)
    else:
        reqs = _upload_requests(synth.make_request_set(1003 + rank, args.requests), dev)
    for r in reqs:
        r["G"] = cbct.cbct_geometry_create(r["geom"])
    stream = torch.cuda.current_stream()
    batch = [dict(geom=r["G"], Y=r["Y_dev"], mu=r["mu"], iters=r["iters"], levels=r["levels"], f_out=r["f_dev"])
             for r in reqs]
    for _ in range(max(1, args.warmup // 3)):
        _sequential(cbct, reqs, stream)
        cbct.cbct_reconstruct_batch(batch, use_graphs=True)
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if rank == 0 else None
    barrier(world)
    seq_s, bat_s = [], []
    for _ in range(args.steps):
        seq_s.append(sum(_sequential(cbct, reqs, stream)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cbct.cbct_reconstruct_batch(batch, use_graphs=True)
        e1.record(stream)
        e1.synchronize()
        bat_s.append(e0.elapsed_time(e1) / 1e3)
    barrier(world)
    clocks = sampler.stop() if sampler else None
    seq_t = max_over_ranks(sum(seq_s), world)
    bat_t = max_over_ranks(sum(bat_s), world)
    n = world * args.steps * len(reqs)
    if rank == 0:
        line = {"mode": "batch", "metric": "reconstructions/s", "value": n / bat_t, "unit": "recon/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * bat_t / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded ellipsoid phantoms, analytic line integrals, Poisson/log noise)",
                "config": {"workload": _request_text(reqs), "step": "all requests once", "graphs": True,
                           "parallelism": f"replicas x{world}"},
                "one_at_a_time": {"value": n / seq_t, "unit": "recon/s", "ms_per_step": 1e3 * seq_t / args.steps},
                "batch_speedup": seq_t / bat_t, "clocks": clocks}
        print(json.dumps(line), flush=True)


def _fifo_latencies(arrivals, service):
    """Latencies of a one-at-a-time FIFO queue with the given arrival and service times."""
    free, out = 0.0, []
    for a, s in zip(arrivals, service):
        start = max(a, free)
        free = start + s
        out.append(free - a)
    return out


def run_serve(args, world, rank, local):
    import torch

    from paper_1002_3675_b300 import cbct

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(1004 + rank)
    if args.mix == "clinical":
        # the medium and large workloads (20, 30 and 40 views), drawn uniformly
        names = ["medium", "large20", "large30", "large"]
        cases = []
        for nm in names:
            c = synth.make_case(nm)
            cfg = synth.CONFIGS[nm]
            cases.append(dict(geom=c["geom"], Y=c["Y"], mu=cfg["mu"], levels=cfg["levels"], iters=cfg["iters"]))
        base = _upload_requests(cases, dev)
        n = args.serve_requests
        order = [int(q) for q in rng.integers(0, len(base), size=n)]
        text = (f"{n} requests drawn uniformly from the medium workload and the large one at 20, 30 and 40 views "
                f"({', '.join(names)})")
    elif args.mix == "small":
        base = _upload_requests(_small_requests(8, 1006 + rank), dev)
        n = args.serve_requests
        order = [q % len(base) for q in range(n)]
        text = _request_text(base) + f" (8 small-workload scans); {n} arrivals cycling through them"
    else:
        base = _upload_requests(synth.make_request_set(1003 + rank, args.requests), dev)
        n = args.serve_requests
        order = [q % len(base) for q in range(n)]
        text = _request_text(base) + f"; {n} arrivals cycling through them"
    for r in base:
        r["G"] = cbct.cbct_geometry_create(r["geom"])
    stream = torch.cuda.current_stream()
    _sequential(cbct, base, stream)
    service = dict(enumerate(_sequential(cbct, base, stream)))
    mean_s = statistics.mean(service[q] for q in order)
    rate = args.load / mean_s                     # arrivals/s at the chosen fraction of one-at-a-time capacity
    gaps = rng.exponential(1.0 / rate, size=n)
    srv = cbct.Server(args.budget_gb << 30, args.slots, use_graphs=True)
    # warm-up: every geometry once, so resident tables and graphs exist
    for r in base:
        srv.wait(srv.submit(r["geom"], r["Y_dev"], r["mu"], r["iters"], r["levels"], r["f_dev"]), 600000)
    outs = [torch.empty_like(base[q]["f_dev"]) for q in order]
    sampler = ClockSampler(local) if rank == 0 else None
    barrier(world)
    t0 = time.perf_counter()
    tickets, arrivals = [], []
    next_t = t0
    for q, gap, f in zip(order, gaps, outs):
        next_t += gap
        while True:
            d = next_t - time.perf_counter()
            if d <= 0:
                break
            time.sleep(min(d, 0.002))
        r = base[q]
        arrivals.append(time.perf_counter() - t0)
        tickets.append(srv.submit(r["geom"], r["Y_dev"], r["mu"], r["iters"], r["levels"], f))
    res = [srv.wait(t, 600000) for t in tickets]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(world)
    clocks = sampler.stop() if sampler else None
    stats = srv.stats()
    srv.close()
    lat = [r["latency_s"] for r in res]
    fifo = _fifo_latencies(arrivals, [service[q] for q in order])
    wall = max_over_ranks(wall, world)
    if rank == 0:
        pct = lambda xs, p: float(np.percentile(np.asarray(xs), p))  # noqa: E731
        line = {"mode": "serve", "metric": "reconstructions/s", "value": world * n / wall, "unit": "recon/s",
                "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * wall,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded ellipsoid phantoms, analytic line integrals, Poisson/log noise)",
                "config": {"workload": text, "arrivals": f"Poisson, {rate:.2f}/s "
                           f"({args.load:.2f} x one-at-a-time capacity)", "slots": args.slots,
                           "hbm_budget_gb": args.budget_gb, "graphs": True, "parallelism": f"replicas x{world}"},
                "latency_s": {"p50": pct(lat, 50), "p90": pct(lat, 90), "p99": pct(lat, 99), "max": max(lat)},
                "fifo_one_at_a_time_latency_s": {"p50": pct(fifo, 50), "p90": pct(fifo, 90), "p99": pct(fifo, 99),
                                                 "max": max(fifo)},
                "mean_service_s": mean_s, "server_busy_s": stats["busy_s"], "clocks": clocks}
        print(json.dumps(line), flush=True)


def run_vcycle(args, world, rank, local):
    """V-cycles against the cascade on the same workload: time and the energy of Eq. 1
    each reaches (float64 energies from the library)."""
    import torch

    from paper_1002_3675_b300 import cbct

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = synth.CONFIGS[args.workload]
    case = synth.make_case(args.workload)
    G = cbct.cbct_geometry_create(case["geom"])
    levels, iters, mu = cfg["levels"], cfg["iters"], cfg["mu"]
    Y = torch.tensor(np.asarray(case["Y"], dtype=np.float32), device=dev)
    f = torch.empty((cfg["vol"][2], cfg["vol"][1], cfg["vol"][0]), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    eps = 2e-5 / min(case["geom"]["hx"], case["geom"]["hy"], case["geom"]["hz"])
    runs = {"vcycle": dict(iters=args.cycles, mg_cycle=1, mg_pre=2, mg_post=2, mg_coarse=10),
            "cascade": dict(iters=iters)}
    out = {}
    for name, kw in runs.items():
        for _ in range(args.warmup):
            cbct.cbct_reconstruct(G, Y, mu, levels=levels, f_out=f, reuse_lambda=True, **kw)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cbct.cbct_reconstruct(G, Y, mu, levels=levels, f_out=f, reuse_lambda=True, **kw)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        E = cbct.cbct_energy(G, Y, f, mu, eps)
        out[name] = {"ms": statistics.median(ms), "energy": float(E[0]), **kw}
    if rank == 0:
        v = out["vcycle"]
        line = {"mode": "vcycle", "metric": "V-cycles/s", "value": args.cycles / (v["ms"] / 1e3), "unit": "cycle/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": v["ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded ellipsoid phantom, analytic line integrals, Poisson/log noise)",
                "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                           "beta": "auto per level, lambda cached across steps"},
                "vcycle": v, "cascade": out["cascade"]}
        print(json.dumps(line), flush=True)


def run_kernels(args, world, rank, local):
    """Profiler target: `--steps` Algorithm A1 iterations on the finest level of the
    workload at its full size, with a fixed beta (no power iteration), so that the
    k-th launch of each kernel is the k-th iteration's.  Prints the ms per iteration."""
    import torch

    from paper_1002_3675_b300 import cbct

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = synth.CONFIGS[args.workload]
    case = synth.make_case(args.workload)
    G = cbct.cbct_geometry_create(case["geom"])
    mu = cfg["mu"]
    Y = torch.tensor(np.asarray(case["Y"], dtype=np.float32), device=dev)
    f = torch.zeros((cfg["vol"][2], cfg["vol"][1], cfg["vol"][0]), dtype=torch.float32, device=dev)
    g = case["geom"]
    eps = 2e-5 / min(g["hx"], g["hy"], g["hz"])
    beta = 10.0 * mu * 1e3  # fixed: the step size does not change the work of an iteration
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cbct.cbct_fbs(G, Y, mu, beta, eps, 10, 0, args.steps, f, tv_mode=args.tv_mode)
    e1.record(stream)
    e1.synchronize()
    if rank == 0:
        ms = e0.elapsed_time(e1)
        print(json.dumps({"mode": "kernels", "workload": args.workload, "iterations": args.steps,
                          "ms_per_iteration": ms / max(args.steps, 1)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="medium", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-quality", action="store_true", help="skip the ground-truth comparison (voxelisation)")
    ap.add_argument("--mode", default="step", choices=["step", "batch", "serve", "vcycle", "kernels"],
                    help="kernels: --steps single-level iterations at full size (a profiler target)")
    ap.add_argument("--cycles", type=int, default=10, help="vcycle: V-cycles per step")
    ap.add_argument("--tv-mode", type=int, default=0, choices=[0, 1], help="E1: 0 isotropic, 1 anisotropic")
    ap.add_argument("--sino-fp16", action="store_true", help="keep the projection data in half precision")
    ap.add_argument("--adjoint-mode", type=int, default=0, choices=[0, 1],
                    help="step-1 adjoint: 0 exact transpose, 1 Eq. 2 interpolation")
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--load", type=float, default=0.8, help="serve: arrival rate / one-at-a-time capacity")
    ap.add_argument("--slots", type=int, default=16, help="serve: slots (one per distinct scan geometry keeps all resident)")
    ap.add_argument("--budget-gb", type=int, default=150)
    ap.add_argument("--mix", default="clinical", choices=["clinical", "batch16", "small"],
                    help="serve: request mix (medium/large workloads, or the 16 heterogeneous requests)")
    ap.add_argument("--serve-requests", type=int, default=40, help="serve: arrivals")
    ap.add_argument("--batch-mix", default="hetero", choices=["hetero", "small"],
                    help="batch: the 16 heterogeneous requests, or --requests copies of the small workload")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.mode == "batch":
        run_batch(args, world, rank, local)
    elif args.mode == "serve":
        run_serve(args, world, rank, local)
    elif args.mode == "vcycle":
        run_vcycle(args, world, rank, local)
    elif args.mode == "kernels":
        run_kernels(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
