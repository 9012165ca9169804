"""Benchmark: FBS iterations/s of the full multigrid reconstruction on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload large]
    python -m torch.distributed.run --nproc-per-node N ... bench.py --gpus N

A step is one complete ``cbct_reconstruct`` call (Algorithm A1 on every multigrid
level: forward projection + residual, adjoint gather + gradient step, M TV-prox
sweeps with f >= 0, float64 energies; the automatic beta's power iterations; the
2x2 data binning and the prolongations) on seeded synthetic data of the workload's
shape.  The default workload is the large one: 512x512x96 voxels, 40 views of
512x384, 3 levels x 50 iterations.  Inputs are resident in HBM when the timed region
starts; L2 is flushed (256 MiB write) between steps, outside the timed events.  The
timed steps carry no per-launch events (one event pair per step and per level); the
per-kernel split and the roofline come from a separate pass of the same steps.  Each
GPU runs independent reconstructions (no data-path collective; weak scaling).

Prints one JSON line.  Besides ``value`` (FBS iterations of every level per second of
whole reconstructions) it carries ``recon_s`` and ``finest_fbs_iter_s`` (the finest
level's iterations alone), and at N = 1 a ``serve`` block: 200 seeded Poisson arrivals
over the medium workload and the large one at 20, 30 and 40 views, served by the
continuous-batching server at 0.5, 0.8 and 1.0 x the one-at-a-time capacity, with
p50/p99 latency against a one-at-a-time FIFO queue fed the same arrivals.

``--impl reference`` times the FP64 CPU oracle on the host cores in the same unit: FBS
iterations per second with every level weighted as in a reconstruction (levels /
the sum over levels of one iteration's time), each step one iteration of one level,
the steps cycling through the levels.

Other modes print their own line:

* ``--mode batch``: 16 heterogeneous requests (six volume sizes from 128^3 to
  384x384x64, 20-60 views, random start angles, 2 levels x 30 iterations), run one at
  a time through ``cbct_reconstruct`` and together through ``cbct_reconstruct_batch``;
  ``--batch-mix small --requests 32`` takes 32 requests of the small workload instead.
* ``--mode serve``: the serving block alone (``--serve-loads``, ``--serve-requests``,
  ``--mix batch16`` for the 16 requests above, ``--mix small`` for small scans).
* ``--mode vcycle``: V-cycles (mg_cycle 1) against the cascade on the workload: time
  per reconstruction and the energy of Eq. 1 each reaches.
* ``--mode kernels``: a profiler target (finest-level iterations with a fixed beta;
  with ``--adjoint-mode 1`` through the Eq. 2 adjoint).
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
# Normalised rate of the projector and the adjoint: lane-operations per nonzero of the
# system matrix.  The primary basis is a flat 5 per nonzero for both operators (a
# Siddon step: next crossing, length, accumulate, advance; the floor the scope table
# of the measurement plan states).  The secondary basis counts what an exact-length
# gather needs per nonzero: adjoint 8 (two z-crossings: 2 sub + 2 mul, clip: 1 max +
# 1 min, length: 1 sub, accumulate: 1 fma), projector 4 (next crossing: 1 min,
# length: 1 sub, accumulate: 1 fma, advance: 1 fma).  Neither kernel does per-nonzero
# work (running slice integrals, a plane sweep over running sums), so both are
# normalised rates, not floors of these kernels.
OPS_PER_NNZ_PLAN = 5.0
OPS_PER_NNZ = {"backproject": 8.0, "project": 4.0}
# Sources of each timed kernel; the DRAM traffic recorded in profiles/ counts only while
# they are unchanged since the capture.
KERNEL_SOURCES = {
    "backproject": ("k_backproject", ["k_backproject.cu", "bp_tile.cuh"]),
    "project": ("k_project", ["k_project.cu", "project_tile.cuh"]),
    "tv": ("k_tv_x", ["k_tv.cu", "tv_tile.cuh", "tv_xmarch.cuh"]),
}


def profile_fields(kernel, workload):
    """Figures of the committed ncu summary of a kernel on a workload (DRAM and L2 bytes
    per operation, issue activity), or {} when there is no summary or the kernel's
    sources changed since it was taken."""
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
        return {}
    s = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    if not s or s.group(1) != h.hexdigest()[:16]:
        return {}
    out = {}
    for key, conv in (("traffic_bytes_per_launch", int), ("l2_bytes_per_launch", int),
                      ("issue_active_pct", float)):
        m = re.search(key + r":\s*([0-9.]+)", text)
        if m:
            out[key] = conv(m.group(1))
    return out


def profile_traffic(kernel, workload):
    return profile_fields(kernel, workload).get("traffic_bytes_per_launch")


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


def _oracle_levels(case, levels):
    """Per-level oracle inputs of the cascade: level geometry, 2x2-binned data and a
    fixed beta of the right size (beta does not change the work of an iteration)."""
    import oracle
    g = case["geom"]
    Ys = [np.asarray(case["Y"], dtype=np.float64)]
    for _ in range(1, levels):
        Ys.append(oracle.restrict_sino(Ys[-1]))
    out = []
    for l in range(levels):
        lg = oracle.level_geom(g, l)
        out.append(dict(geom=lg, Y=Ys[l], beta=1.05 * oracle.gamma(lg, case["mu"]) * 1.6e4 / 4 ** l,
                        eps=oracle.default_eps(lg)))
    return out


def oracle_iteration_s(case, lvl):
    """Seconds of one Algorithm A1 iteration of the oracle (P, P^T, 10 prox sweeps) on
    one level, from f = 0."""
    import oracle
    g = lvl["geom"]
    f0 = np.zeros((g["nz"], g["ny"], g["nx"]))
    t0 = time.perf_counter()
    oracle.fbs(g, lvl["Y"], case["mu"], lvl["beta"], lvl["eps"], 10, 1, f0=f0)
    return time.perf_counter() - t0


def oracle_level_rate(case, levels, steps, warmup):
    """The oracle's FBS iterations/s with every level weighted as in a reconstruction
    (the same number of iterations per level): levels / sum_l t_l, t_l the mean time of
    one iteration on level l.  Step q runs one iteration on level q mod levels (at
    least one step per level); the warm-up steps run on the coarsest level."""
    import oracle
    lv = _oracle_levels(case, levels)
    for _ in range(warmup):
        oracle_iteration_s(case, lv[-1])
    per = [[] for _ in range(levels)]
    n = max(steps, levels)
    for q in range(n):
        per[q % levels].append(oracle_iteration_s(case, lv[q % levels]))
    t_l = [statistics.mean(x) for x in per]
    return {"value": levels / sum(t_l), "level_s": t_l, "steps": n, "total_s": sum(map(sum, per)),
            "cores": oracle.num_threads()}


def config_of(args, cfg, world):
    """The `config` object of the line, the same in both arms (what each arm did beyond
    it goes to the line's `run` object)."""
    return {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}", "inner_iters": 10,
            "parallelism": f"replicas x{world}",
            "variant": {"tv_mode": ["isotropic", "anisotropic"][args.tv_mode],
                        "adjoint": ["exact transpose", "Eq. 2 interpolation"][args.adjoint_mode],
                        "data_storage": "float16" if args.sino_fp16 else "float32"},
            "fbs_iterations_per_step": cfg["levels"] * cfg["iters"],
            "unit_note": "FBS iterations per second with every multigrid level weighted as in one "
                         "reconstruction (the same number of iterations on each level)"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    cfg = synth.CONFIGS[args.workload]
    case = synth.make_case(args.workload)
    r = oracle_level_rate(case, cfg["levels"], args.steps, args.warmup)
    sample = (f"{r['steps']} steps, each one Algorithm A1 iteration (P, P^T, 10 prox sweeps, from f = 0, fixed "
              f"beta) on one level of the {cfg['levels']}-level cascade in turn; value = levels / sum of the "
              f"per-level mean times ({', '.join(f'{t:.3f}' for t in r['level_s'])} s, finest first); "
              f"warm-up on the coarsest level")
    config = config_of(args, cfg, world)
    run = {"beta": "fixed per level (no power iteration)", "host_cores": os.cpu_count(),
           "ranks": "the FP64 oracle on the host cores (rank 0 only); n_gpus is the launch's rank count"}
    line = {"impl": "reference", "metric": "FBS iterations/s", "value": r["value"], "unit": "iter/s",
            "n_gpus": world, "steps": r["steps"], "warmup": args.warmup, "ms_per_step": 1e3 * r["total_s"] / r["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded ellipsoid phantom, analytic line integrals, Poisson/log noise)",
            "config": config, "run": run,
            "finest_fbs_iter_s": 1.0 / r["level_s"][0],
            "cpu_baseline": {"value": r["value"], "unit": "iter/s", "cores": r["cores"], "cpu_model": cpu_model(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": r["value"], "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    # a stream of its own: the library replays each level's iteration as a CUDA graph
    # (graphs need a stream other than the legacy default one)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        res = _gpu_steps(args, cbct, G, Y, Y_host, f, f_host, flush, stream, levels, iters, mu, world,
                         local if rank == 0 else None)
    if rank != 0:
        return
    _gpu_line(args, cbct, torch, dev, G, case, cfg, Y, Y_host, f, f_host, res, world)


def _gpu_steps(args, cbct, G, Y, Y_host, f, f_host, flush, stream, levels, iters, mu, world, clock_gpu):
    import torch
    graphs = not args.no_graphs

    def step(**kw):
        return cbct.cbct_reconstruct(G, Y, mu, iters, levels, f_out=f, tv_mode=args.tv_mode,
                                     adjoint_mode=args.adjoint_mode, sino_fp16=args.sino_fp16, use_graphs=graphs,
                                     **kw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-resident timed region: one event pair per step (and per level) -------
    sampler = ClockSampler(clock_gpu) if clock_gpu is not None else None
    barrier(world)
    torch.cuda.synchronize()
    step_ms, level_ms = [], [0.0] * levels
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = step(level_times=True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        level_ms = [a + b for a, b in zip(level_ms, info["level_ms"])]
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    tot_ms = max_over_ranks(sum(step_ms), world)
    fin_ms = max_over_ranks(level_ms[0], world)

    # ---- end to end through the C ABI with host buffers ---------------------------
    barrier(world)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Y.copy_(Y_host, non_blocking=True)
        step()
        f_host.copy_(f, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_tot = max_over_ranks(sum(e2e_ms), world)

    # ---- every kernel class timed launch by launch: a separate pass of the same steps,
    #      the power iterations in level order so that no two streams share the event
    #      windows (per-launch events keep the graphs off in this pass) ------------------
    split_ms, split_n, kms_f, kl_f = {}, {}, {}, {}
    n0 = cbct.cbct_kernel_launch_count()
    for _ in range(args.steps):
        flush.fill_(1)
        _, info = step(kernel_times=True, kernel_mask=0, serial_power=True)
        for src, dst in ((info["kernel_ms"], split_ms), (info["kernel_launches"], split_n),
                         (info["kernel_ms_finest"], kms_f), (info["kernel_launches_finest"], kl_f)):
            for k, v in src.items():
                dst[k] = dst.get(k, 0) + v
    torch.cuda.synchronize()
    # kernels per step (the timed steps launch the same kernels; their graph replays do
    # not pass through the library's launch sites, so they are counted here)
    launches_per_step = (cbct.cbct_kernel_launch_count() - n0) / args.steps

    # ---- the same steps with lambda_max(P^T P) cached per geometry (reported beside) --
    step(reuse_lambda=True)   # fills the cache
    torch.cuda.synchronize()
    cached_ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(reuse_lambda=True)
        e1.record(stream)
        e1.synchronize()
        cached_ms.append(e0.elapsed_time(e1))
    cached_tot = max_over_ranks(sum(cached_ms), world)
    return dict(tot_ms=tot_ms, fin_ms=fin_ms, level_ms=level_ms, e2e_tot=e2e_tot, split_ms=split_ms,
                split_n=split_n, kms_f=kms_f, kl_f=kl_f, launches_per_step=launches_per_step,
                cached_tot=cached_tot, clocks=clocks, graphs=graphs)


def _gpu_line(args, cbct, torch, dev, G, case, cfg, Y, Y_host, f, f_host, res, world):
    levels, iters, mu = cfg["levels"], cfg["iters"], cfg["mu"]
    tot_ms, split_ms, split_n, kms_f, kl_f = res["tot_ms"], res["split_ms"], res["split_n"], res["kms_f"], res["kl_f"]
    clocks = res["clocks"]
    n_iter = levels * iters
    value = world * args.steps * n_iter / (tot_ms / 1e3)

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
    # rates from the finest level's Algorithm A1 iterations (they run after every power
    # iteration has finished, so nothing shares their event windows)
    units_f = {k: nnz[0] * iters for k in ("project", "backproject")}
    per_kernel = {}
    for k in ("project", "backproject"):
        t = kms_f[k] / 1e3
        per_kernel[k] = {"ms_per_step": split_ms[k] / args.steps, "launches_per_step": split_n[k] / args.steps,
                         "finest_fbs_ms_per_step": kms_f[k] / args.steps,
                         "finest_fbs_launches_per_step": kl_f[k] / args.steps,
                         "ms_per_operation": kms_f[k] / (args.steps * iters)}
        if k == "backproject" and args.adjoint_mode == 1:
            per_kernel[k]["note"] = "Eq. 2 adjoint in the FBS iterations: no nonzero-based rate"
            continue
        per_kernel[k]["gnnz_per_s"] = units_f[k] * args.steps / t / 1e9
        per_kernel[k]["alu_tops_plan_basis"] = units_f[k] * args.steps * OPS_PER_NNZ_PLAN / t / 1e12
        per_kernel[k]["alu_tops_kernel_basis"] = units_f[k] * args.steps * OPS_PER_NNZ[k] / t / 1e12
        pf = profile_fields(k, args.workload)
        if "l2_bytes_per_launch" in pf:
            per_kernel[k]["l2_gbs"] = pf["l2_bytes_per_launch"] / (per_kernel[k]["ms_per_operation"] / 1e3) / 1e9
        if "issue_active_pct" in pf:
            per_kernel[k]["issue_active_pct"] = pf["issue_active_pct"]
    nvox = [np.prod([(n + (1 << l) - 1) >> l for n in cfg["vol"]]) for l in range(levels)]
    tv_bytes = sum(12.0 * v * iters * 10 for v in nvox) * args.steps   # read f, read g, write f per sweep
    per_kernel["tv"] = {"ms_per_step": split_ms["tv"] / args.steps,
                        "gbs": tv_bytes / (split_ms["tv"] / 1e3) / 1e9, "launches_per_step": split_n["tv"] / args.steps,
                        "note": "HBM-equivalent rate: 12 B per voxel per prox sweep (10 sweeps per iteration), "
                                "whatever the number of sweeps fused per launch"}
    pf_tv = profile_fields("tv", args.workload)
    if pf_tv:
        per_kernel["tv"]["profile"] = {k: v for k, v in pf_tv.items()}
    timing = ("CUDA events on the launching stream around every operation of the class, in a separate pass of "
              "the same steps (the headline steps carry no per-launch events); rates from the finest level's "
              "Algorithm A1 iterations, which run with nothing beside them")
    if dom in ("project", "backproject"):
        pk = per_kernel[dom]
        ach = pk["alu_tops_plan_basis"]
        pf = profile_fields(dom, args.workload)
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "Tlane-op/s",
                "frac": ach / alu_peak, "traffic": pf.get("traffic_bytes_per_launch"),
                "launch_ms": pk["ms_per_operation"], "timing": timing,
                "basis": f"{OPS_PER_NNZ_PLAN:.0f} lane-ops per nonzero (the measurement plan's floor) x the "
                         f"finest level's exact nnz ({nnz[0]}) per operation; peak = {sm_count} SMs x 128 FP32 "
                         f"lanes x {clock_mhz:.0f} MHz (median SM clock in the timed region). Normalised rate: "
                         "the kernel does no per-nonzero work",
                "basis_survey": {"ops_per_nnz": OPS_PER_NNZ_PLAN, "frac": ach / alu_peak},
                "basis_kernel": {"ops_per_nnz": OPS_PER_NNZ[dom],
                                 "frac": pk["alu_tops_kernel_basis"] / alu_peak},
                "l2_gbs": pk.get("l2_gbs"), "issue_active_pct": pk.get("issue_active_pct"),
                "operation": "one projection (its slab launches)" if dom == "project"
                             else "one adjoint (column running sums + gather)"}
    else:
        ach = per_kernel["tv"]["gbs"]
        roof = {"kernel": "tv", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": profile_traffic("tv", args.workload), "timing": timing}
    roof["peak_source"] = peak_kind

    # ---- CPU baseline: the oracle on a bounded sample, in the same unit ---------------
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        r = oracle_level_rate(case, levels, levels, 0)
        cpu = {"value": r["value"], "unit": "iter/s", "cores": r["cores"], "cpu_model": cpu_model(), "kind": "oracle",
               "finest_fbs_iter_s": 1.0 / r["level_s"][0],
               "sample": f"one Algorithm A1 iteration (P, P^T, 10 prox sweeps) on each of the {levels} levels of "
                         f"the same workload, FP64 C oracle with OpenMP, fixed beta, no power iteration; value = "
                         f"levels / sum of the per-level times ({', '.join(f'{t:.3f}' for t in r['level_s'])} s)"}

    # ---- per-iteration fractions (algorithmic HBM bytes and the composite floor) -------
    s_bytes = 2 if args.sino_fp16 else 4
    dims = [cbct.cbct_level_dims(G, l) for l in range(levels)]
    nv_l = [d[0] * d[1] * d[2] for d in dims]
    nr_l = [len(case["geom"]["angles"]) * d[3] * d[4] for d in dims]
    b_fbs = sum(24 * v + (8 + s_bytes) * r for v, r in zip(nv_l, nr_l)) * iters       # per step
    b_pow = sum(8 * v + 8 * r for v, r in zip(nv_l, nr_l)) * K_pi
    bw = peaks["hbm_gbs"] * 1e9
    t_step = tot_ms / args.steps / 1e3
    floor_s = {"project": units["project"] * OPS_PER_NNZ_PLAN / (alu_peak * 1e12),
               "backproject": units["backproject"] * OPS_PER_NNZ_PLAN / (alu_peak * 1e12),
               "tv": sum(12.0 * v for v in nv_l) * iters / bw}
    per_iter = {"hbm_bytes_per_fbs_iteration_finest": 24 * nv_l[0] + (8 + s_bytes) * nr_l[0],
                "literal_hbm_frac": (b_fbs + b_pow) / (t_step * bw),
                "composite_frac": sum(floor_s.values()) / t_step,
                "floor_ms_per_step": {k: v * 1e3 for k, v in floor_s.items()},
                "basis": "literal: (24 Nv + (8+s) Nr) bytes per FBS iteration and (8 Nv + 8 Nr) per power "
                         "iteration over the step time at the measured HBM bandwidth; composite: the sum of "
                         "the per-class floors (P and P^T: nonzeros x 5 lane-ops / FP32 issue peak; TV: 12 B "
                         "per voxel per Algorithm A1 iteration, all sweeps fused, / HBM) over the step time"}

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

    # ---- serving (continuous batching) on the medium/large mix -------------------------
    serve = None
    if world == 1 and not args.no_serve:
        loads = [float(x) for x in args.serve_loads.split(",")]
        serve = serve_measure(args, 0, dev, loads, args.serve_requests, args.mix)

    config = config_of(args, cfg, world)
    run = {"beta": "auto per level (30 power iterations, recomputed every step)",
           "l2": "flushed between steps (256 MiB write, untimed)",
           "graphs": "each level's Algorithm A1 iteration replayed as a captured CUDA graph" if res["graphs"]
           else "off"}
    line = {
        "metric": "FBS iterations/s", "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ellipsoid phantom, analytic line integrals, Poisson/log noise); "
                "stands in for the paper's NCAT/CatPhan data",
        "config": config, "run": run,
        "recon_s": tot_ms / args.steps / 1e3,
        "finest_fbs_iter_s": world * args.steps * iters / (res["fin_ms"] / 1e3),
        "level_ms_per_step": [v / args.steps for v in res["level_ms"]],
        "e2e": {"value": world * args.steps * n_iter / (res["e2e_tot"] / 1e3), "unit": "iter/s",
                "h2d_bytes_per_step": int(Y_host.numel() * 4), "d2h_bytes_per_step": int(f_host.numel() * 4)},
        "lambda_cached": {"value": world * args.steps * n_iter / (res["cached_tot"] / 1e3), "unit": "iter/s",
                          "ms_per_step": res["cached_tot"] / args.steps,
                          "note": "beta's power iterations reused from an earlier call on the same geometry"},
        "roofline": roof,
        "kernels": per_kernel,
        "kernel_ms_per_step": {k: v / args.steps for k, v in split_ms.items()},
        "kernel_split_note": "kernel_ms_per_step: every launch timed with CUDA events in a separate pass of the "
                             "same steps, the power iterations in level order (serial_power)",
        "gpu_launches": int(round(res["launches_per_step"] * args.steps)),
        "gpu_launches_note": "kernels per step counted by the library's launch sites in the separate pass "
                             "(the same kernels as the timed steps, whose per-level graphs replay them) x steps",
        "per_iteration": per_iter,
        "quality": quality,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if serve is not None:
        line["serve"] = serve
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
    # (NVTX ranges name the two halves of a timed step, so that a profiler can take the
    # launches of one of them: ncu --nvtx --nvtx-include "batched_step/")
    for _ in range(args.steps):
        torch.cuda.nvtx.range_push("sequential_step")
        seq_s.append(sum(_sequential(cbct, reqs, stream)))
        torch.cuda.nvtx.range_pop()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("batched_step")
        e0.record(stream)
        cbct.cbct_reconstruct_batch(batch, use_graphs=True)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
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


def _serve_base(args, rank, dev, mix):
    """The request kinds of a serving mix (uploaded) and a description."""
    if mix == "clinical":
        # the medium and large workloads (20, 30 and 40 views), drawn uniformly
        names = ["medium", "large20", "large30", "large"]
        cases = []
        for nm in names:
            c = synth.make_case(nm)
            cfg = synth.CONFIGS[nm]
            cases.append(dict(geom=c["geom"], Y=c["Y"], mu=cfg["mu"], levels=cfg["levels"], iters=cfg["iters"]))
        return _upload_requests(cases, dev), ("requests drawn uniformly from the medium workload and the large one "
                                              f"at 20, 30 and 40 views ({', '.join(names)})"), True
    if mix == "small":
        base = _upload_requests(_small_requests(8, 1006 + rank), dev)
        return base, _request_text(base) + " (8 small-workload scans), arrivals cycling through them", False
    base = _upload_requests(synth.make_request_set(1003 + rank, args.requests), dev)
    return base, _request_text(base) + ", arrivals cycling through them", False


def serve_measure(args, rank, dev, loads, n, mix):
    """Continuous-batching server against a one-at-a-time FIFO queue: n seeded Poisson
    arrivals at each load (a fraction of the one-at-a-time capacity).  Returns a dict."""
    import torch

    from paper_1002_3675_b300 import cbct

    base, text, drawn = _serve_base(args, rank, dev, mix)
    for r in base:
        r["G"] = cbct.cbct_geometry_create(r["geom"])
    stream = torch.cuda.current_stream()
    _sequential(cbct, base, stream)
    service = dict(enumerate(_sequential(cbct, base, stream)))
    srv = cbct.Server(args.budget_gb << 30, args.slots, use_graphs=True)
    # warm-up: every geometry once, so resident tables and graphs exist
    for r in base:
        srv.wait(srv.submit(r["geom"], r["Y_dev"], r["mu"], r["iters"], r["levels"], r["f_dev"]), 600000)
    pct = lambda xs, p: float(np.percentile(np.asarray(xs), p))  # noqa: E731
    out = {"workload": f"{n} arrivals per load, " + text, "slots": args.slots, "hbm_budget_gb": args.budget_gb,
           "graphs": True, "service_s": {str(q): service[q] for q in service}, "loads": []}
    for li, load in enumerate(loads):
        rng = np.random.default_rng(1004 + rank + 1000 * li)
        order = [int(q) for q in rng.integers(0, len(base), size=n)] if drawn else [q % len(base) for q in range(n)]
        mean_s = statistics.mean(service[q] for q in order)
        rate = load / mean_s                    # arrivals/s at this fraction of one-at-a-time capacity
        gaps = rng.exponential(1.0 / rate, size=n)
        outs = [torch.empty_like(base[q]["f_dev"]) for q in order]
        busy0 = srv.stats()["busy_s"]
        t0 = time.perf_counter()
        tickets, arrivals = [], []
        next_t = t0
        for q, gap, fo in zip(order, gaps, outs):
            next_t += gap
            while True:
                d = next_t - time.perf_counter()
                if d <= 0:
                    break
                time.sleep(min(d, 0.002))
            r = base[q]
            arrivals.append(time.perf_counter() - t0)
            tickets.append(srv.submit(r["geom"], r["Y_dev"], r["mu"], r["iters"], r["levels"], fo))
        res = [srv.wait(t, 600000) for t in tickets]
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        lat = [r["latency_s"] for r in res]
        fifo = _fifo_latencies(arrivals, [service[q] for q in order])
        fifo_wall = max(a + l for a, l in zip(arrivals, fifo))
        out["loads"].append({
            "load": load, "arrival_rate_per_s": rate, "arrivals": n, "wall_s": wall,
            "recon_per_s": n / wall, "fifo_recon_per_s": n / fifo_wall,
            "latency_s": {"p50": pct(lat, 50), "p90": pct(lat, 90), "p99": pct(lat, 99), "max": max(lat)},
            "fifo_one_at_a_time_latency_s": {"p50": pct(fifo, 50), "p90": pct(fifo, 90), "p99": pct(fifo, 99),
                                             "max": max(fifo)},
            "mean_service_s": mean_s, "server_busy_s": srv.stats()["busy_s"] - busy0})
    srv.close()
    out["note"] = ("FIFO: a zero-overhead one-at-a-time queue replayed with the same arrival times and the "
                   "measured cbct_reconstruct service time of each request")
    return out


def run_serve(args, world, rank, local):
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    loads = [float(x) for x in args.serve_loads.split(",")]
    sampler = ClockSampler(local) if rank == 0 else None
    barrier(world)
    t0 = time.perf_counter()
    serve = serve_measure(args, rank, dev, loads, args.serve_requests, args.mix)
    wall = max_over_ranks(time.perf_counter() - t0, world)
    barrier(world)
    clocks = sampler.stop() if sampler else None
    if rank == 0:
        main = serve["loads"][len(loads) // 2]
        line = {"mode": "serve", "metric": "reconstructions/s", "value": world * main["recon_per_s"],
                "unit": "recon/s", "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * wall,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded ellipsoid phantoms, analytic line integrals, Poisson/log noise)",
                "config": {"workload": serve["workload"], "value_at_load": main["load"],
                           "parallelism": f"replicas x{world}"},
                "serve": serve, "clocks": clocks}
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
    if args.adjoint_mode:
        # the Eq. 2 adjoint: one level of the cascade with the same fixed beta
        cbct.cbct_reconstruct(G, Y, mu, args.steps, 1, f_out=f, beta=beta, eps=eps, inner_iters=10,
                              tv_mode=args.tv_mode, adjoint_mode=args.adjoint_mode)
    else:
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
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOAD_TEXT))
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
    ap.add_argument("--slots", type=int, default=16, help="serve: slots (one per distinct scan geometry keeps all resident)")
    ap.add_argument("--budget-gb", type=int, default=150)
    ap.add_argument("--mix", default="clinical", choices=["clinical", "batch16", "small"],
                    help="serve: request mix (medium/large workloads, or the 16 heterogeneous requests)")
    ap.add_argument("--serve-requests", type=int, default=200, help="serve: arrivals per load")
    ap.add_argument("--serve-loads", default="0.5,0.8,1.0",
                    help="serve: arrival rates as fractions of the one-at-a-time capacity")
    ap.add_argument("--no-serve", action="store_true", help="step mode: skip the serving block")
    ap.add_argument("--no-graphs", action="store_true", help="step mode: launch every kernel (no CUDA graphs)")
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
