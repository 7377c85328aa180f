#!/usr/bin/env python3
"""Throughput of the coupled LB-EHD step (MLUPS) and the HBM roofline fraction of its
dominant kernel on B300.

One benchmark step = ``--lb-steps`` coupled lattice Boltzmann time steps (phase moments
and wetting ghosts, Poisson solve, forces, fused collide + stream of all populations,
observable reductions) of the workload, whose state (~350 MB for the 128x64x64 lattice)
is larger than L2, so no L2 flush is needed between steps.

Beside the plain line: the 64-instance batched sweep ("batched") and the adjoint of the
differentiable-control case ("adjoint": forward + backward cost per step against the plain
step of the same schedule).

Arms:
  default            the CUDA library through its C ABI, inputs resident in HBM;
  --impl reference   the FP64 CPU oracle on the host cores (a deliberately slow program;
                     reported as a baseline, not a target).
Multi-GPU (torchrun): independent replicas, one per GPU; no collective on the data path.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Coupled LB-EHD MLUPS, % of HBM roofline; batched/adjoint vs plain on 1 B300"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6400.0

# Algorithmic bytes per fluid-site update of the fused collide kernel (FP32): every
# population read once and written once (3D: 19 + 3*19 + 7 = 83 floats each way), plus the
# site's own fields: Phi_i and Phi_i^{n-1} (24), rho_e and rho_e^{n-1} (8), u read+write (24),
# conduction source read+write (8), potential (4), node class (1).
COLLIDE_BYTES = {3: 83 * 4 * 2 + 24 + 8 + 24 + 8 + 4 + 1, 2: 41 * 4 * 2 + 24 + 8 + 24 + 8 + 4 + 1}
# Whole-step model of the hot path per site update: populations read + written once
# (664 B in 3D), macroscopic fields ~92 B, and ~16 B per Poisson sweep.
STEP_BYTES = {3: (756, 16), 2: (388, 12)}
# DRAM bytes per launch of the collide kernel (dram__bytes_read.sum + dram__bytes_write.sum,
# mean of 2 launches in one ncu capture of the current kernel, summarised under profiles/),
# by workload and autotuned variant. Only these are reported as roofline traffic; a variant
# without a capture of the current kernel reports null.
COLLIDE_TRAFFIC = {("droplet_3d_128x64x64", "staged32x4"): 341.23e6,
                   ("droplet_3d_128x64x64", "staged64x2"): 342.37e6}
# LBEHD_OPT_COLLIDE values
COLLIDE_CHOICES = {"auto": 0, "global": 1, "staged": 2, "staged64x2": 3, "staged16x8": 4}
VARIANT_NAMES = {1: "global", 2: "staged32x4", 3: "staged64x2", 4: "staged16x8"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons, sampled every 50 ms with timestamps from before
    the warm-up to the end of the last timed region; summary(t0, t1) keeps the samples
    taken inside one timed region (host wall-clock seconds)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]
            self.proc = None

    @staticmethod
    def _epoch(stamp):
        import datetime
        try:
            return datetime.datetime.strptime(stamp.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self, t0, t1):
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            t = self._epoch(parts[0])
            if t is None or not (t0 <= t <= t1):
                continue
            try:
                sm.append(float(parts[2]))
                smax = float(parts[3])
            except ValueError:
                continue
            for name, val in zip(names, parts[6:10]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "window_s": round(t1 - t0, 3), "sampler": "nvidia-smi -lms 50"}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(workload, steps, budget_s=None, warm_steps=0, threads=None):
    """Time the FP64 oracle as it stands on the host cores: `warm_steps` untimed coupled
    steps (the first solves start from phi = 0 and take the most CG iterations), then up to
    `steps` timed ones, stopping early once `budget_s` seconds have been spent.
    Returns (MLUPS, timed steps, threads used, seconds)."""
    from oracle import oracle as O
    cores = threads or len(os.sched_getaffinity(0))
    O.set_threads(cores)
    w = workload
    sim = O.OracleSim(w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
    if warm_steps:
        sim.step(warm_steps)
    done, t0 = 0, time.perf_counter()
    while done < steps:
        sim.step(1)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return w.sites * done / dt / 1e6, done, O.get_threads(), dt


def run_reference(args, world, rank):
    """The FP64 oracle on the host cores, on the same workload and metric. One benchmark
    step of this arm is ONE coupled step of the whole lattice (the oracle needs seconds per
    step): --warmup untimed steps, then --steps timed ones (fewer if the time budget
    LBEHD_REF_BUDGET_S runs out first); `steps` and `ms_per_step` report what ran."""
    if rank != 0:
        return
    from paper_2608_12868_b300 import workloads as W
    w = W.WORKLOADS[args.workload]()
    budget = float(os.environ.get("LBEHD_REF_BUDGET_S", "150"))
    mlups, done, cores, dt = cpu_oracle_rate(w, args.steps, budget_s=budget,
                                             warm_steps=args.warmup)
    sample = (f"{done} timed coupled steps (after {args.warmup} untimed) of the full "
              f"{'x'.join(map(str, w.shape[::-1]))} lattice (of {args.steps} requested; "
              f"capped at {budget:.0f} s), FP64, {cores} threads")
    line = {
        "metric": METRIC, "value": mlups, "unit": UNIT, "impl": "reference", "n_gpus": world,
        "steps": done, "warmup": args.warmup, "ms_per_step": dt / done * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "sites": w.sites, "lb_steps_per_step": 1},
        "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_oracle_baselines(args):
    """The CPU baselines of the plan: the FP64 oracle single-threaded and on every host core,
    on the 2D 128x64 workload (all 2000 steps) and on the 3D 128x64x64 workload (its first
    steps). One JSON line per measurement."""
    from paper_2608_12868_b300 import workloads as W
    cores = len(os.sched_getaffinity(0))
    plan = [("droplet_2d_128x64", 2000, 0), ("droplet_3d_128x64x64", args.oracle_3d_steps, 0)]
    for name, steps, warm in plan:
        w = W.WORKLOADS[name]()
        for threads in (1, cores):
            mlups, done, used, dt = cpu_oracle_rate(w, steps, warm_steps=warm, threads=threads)
            print(json.dumps({"oracle_baseline": name, "steps": done, "threads": used,
                              "seconds": dt, "value": mlups, "unit": UNIT}), flush=True)


def run_ours(args, world, rank, local):
    import torch
    from paper_2608_12868_b300 import lbehd
    from paper_2608_12868_b300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.WORKLOADS[args.workload]()
    stream = torch.cuda.Stream(dev)
    mode = {"fixed": lbehd.POISSON_FIXED, "host": lbehd.POISSON_HOST,
            "graph": lbehd.POISSON_GRAPH}[args.poisson]
    sim = lbehd.Simulation(w, stream=stream, device=local, poisson_mode=mode,
                           poisson_fixed_iters=args.fixed_iters,
                           poisson_check_every=args.check_every)
    tuned = None
    if args.collide == "tune":
        sim.step(1)
        variant, tune_ms = sim.autotune(reps=20)
        tuned = {"variant": VARIANT_NAMES[variant],
                 "ms_per_launch": {VARIANT_NAMES[v]: round(t, 5) for v, t in tune_ms.items()}}
    else:
        sim.set_option(lbehd.OPT_COLLIDE, COLLIDE_CHOICES[args.collide])
    L = args.lb_steps
    fluid = int((w.solid == 0).sum())
    clk = ClockSampler(local).start()
    for _ in range(args.warmup):
        sim.step(L)
    torch.cuda.synchronize(dev)
    # keep warming up until the GPU has been busy for ~2 s (clocks and HBM ramp up)
    t_w = time.perf_counter()
    while time.perf_counter() - t_w < args.warmup_seconds:
        sim.step(L)
        torch.cuda.synchronize(dev)
    warm_obs = sim.observe()

    # ---------------- timed region: device time, inputs resident in HBM
    st0 = sim.stats()
    barrier(world)
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_region0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        sim.step(L)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t_region1 = time.time()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    st1 = sim.stats()
    launches = st1["kernels"] - st0["kernels"]
    iters_per_step = (st1["poisson_iters"] - st0["poisson_iters"]) / (L * args.steps)
    obs = sim.observe()
    ms_max = max_over_ranks(world, ms, dev)
    value = w.sites * L * args.steps * world / (ms_max / 1e3) / 1e6

    # ---------------- second timed region of the same length with CUDA events around every
    # launch (eager launches: events cannot sit between the nodes of a replayed graph)
    sim.profile(True)
    torch.cuda.synchronize(dev)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(args.steps):
        sim.step(L)
    pe1.record(stream)
    torch.cuda.synchronize(dev)
    prof_ms = pe0.elapsed_time(pe1)
    prof = sim.profile_read()
    sim.profile(False)

    # ---------------- end to end through the C ABI with host buffers
    Vh = np.ascontiguousarray(w.params.get("V", []), dtype=np.float64)
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.set_electrodes(Vh)      # per-step input: electrode potentials (host -> device)
        sim.step(L)
        sim.observe()               # per-step result: droplet observables (device -> host)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(world, time.perf_counter() - t0, dev)
    e2e = w.sites * L * args.steps * world / e2e_s / 1e6

    # ---------------- roofline of the dominant kernel (fused collide + stream)
    peak, peak_kind = measured_peaks()
    coll_ms, coll_n = prof["collide"]
    coll_avg_s = coll_ms / max(coll_n, 1) / 1e3
    coll_bytes = fluid * COLLIDE_BYTES[w.dim] + w.sites
    achieved = coll_bytes / coll_avg_s / 1e9
    sb, sp = STEP_BYTES[w.dim]
    step_bytes = w.sites * (sb + sp * iters_per_step)
    step_gbs = step_bytes / (ms / 1e3 / (L * args.steps)) / 1e9
    share = {k: round(v[0] / prof_ms, 4) for k, v in prof.items()}

    others = {}
    if args.other_workloads:
        for name, n in (("droplet_2d_128x64", 2000), ("transport_3d_384x128x96", 4000),
                        ("droplet_3d_128x64x64_table1_densities", 2000)):
            others[name] = run_workload_line(args, dev, name, n, peak, peak_kind)
    batched = None
    if args.batched > 0:
        batched = run_batched(args, dev, value / world, peak, peak_kind, clk)
    adjoint = None
    if args.adjoint_segments > 0 and args.adjoint_seg_steps > 0:
        adjoint = run_adjoint(args, dev)
    clk.stop()
    for extra in (batched, adjoint, *others.values()):
        if extra is not None:
            extra["clocks"] = clk.summary(*extra.pop("window"))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mlups, done, cores, dt = cpu_oracle_rate(w, args.cpu_steps, budget_s=args.cpu_seconds,
                                                 warm_steps=1)
        cpu = {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{done} coupled steps of the same lattice after one untimed step, "
                         f"FP64, {dt:.1f} s"}

    if rank == 0:
        clocks = clk.summary(t_region0, t_region1)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": w.name, "sites": w.sites, "fluid_sites": fluid,
                "lb_steps_per_step": L, "lb_steps_before_timed": st0["steps"],
                "parallelism": f"replicas{world}",
                "poisson": f"MG-preconditioned CG on the increment, {args.poisson} convergence",
                "poisson_iters_per_lb_step": iters_per_step,
                "l2": "state (~350 MB) larger than the 126 MB L2; no flush",
                "step_bytes_model_per_site": sb + sp * iters_per_step,
                "step_gbs_model": step_gbs,
                "kernel_time_share_eager_pass": share,
                "eager_pass_ms_per_step": prof_ms / args.steps,
            },
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": COLLIDE_TRAFFIC.get(
                             (w.name, tuned["variant"] if tuned else args.collide)),
                         "kernel": "k_collide (" + (tuned["variant"] if tuned else args.collide)
                                   + ")", "peak_source": peak_kind,
                         "timing": "CUDA events around each k_collide launch over a second "
                                   "timed region of the same length",
                         "bytes_per_launch": coll_bytes},
            "step_roofline": {
                "bytes_per_update": sb + sp * iters_per_step,
                "model": f"{sb} B per site update (populations read + written, fields) + "
                         f"{sp} B per CG iteration x {iters_per_step:.3f} iterations per step",
                "achieved_gbs": step_gbs, "frac_of_measured": step_gbs / peak,
                "frac_of_nominal_8tbs": step_gbs / 8000.0},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": Vh.nbytes,
                    # lbehd_observe reads back the last two steps' 16 observable sums
                    # (FP64), the error flag, the CG scalars (104 B) and the barrier error word
                    "d2h_bytes_per_step": 2 * 16 * 8 + 4 + 104 + 4},
            "gpu_launches": launches,
            "clocks": clocks,
            "autotune": tuned,
            "batched": batched,
            "adjoint": adjoint,
            "other_workloads": others or None,
            "obs_status": obs["status"],
            "mass_drift": float(np.abs(obs["mass"] / warm_obs["mass"] - 1).max()),
        }
        print(json.dumps(line), flush=True)


def run_workload_line(args, dev, name, steps, peak, peak_kind):
    """Throughput of another configuration in the benchmark's launch configuration (step
    graphs, persistent Gauss-law solve, autotuned collide kernel): `steps` coupled steps
    timed with CUDA events after a warm-up, inputs resident. A workload with an electrode
    schedule switches electrodes at its scheduled steps (the switch synchronises, between
    timed chunks)."""
    import torch
    from paper_2608_12868_b300 import lbehd
    from paper_2608_12868_b300 import workloads as W
    w = W.WORKLOADS[name]()
    stream = torch.cuda.Stream(dev)
    sim = lbehd.Simulation(w, stream=stream, device=dev.index, poisson_mode=lbehd.POISSON_GRAPH)
    sim.step(1)
    variant, _ = sim.autotune(reps=5)
    sched = sorted(w.schedule) if len(w.schedule) > 1 else []
    warm = min(args.warmup * 100, 1000)
    sim.step(warm)
    torch.cuda.synchronize(dev)
    t = 1 + warm
    m0 = sim.observe()["mass"]
    st0 = sim.stats()
    # chunks between electrode switches inside the timed window
    cuts = [k for k, _ in sched if t < k < t + steps]
    bounds = [t] + cuts + [t + steps]
    ms = 0.0
    t_region0 = time.time()
    for a, b in zip(bounds[:-1], bounds[1:]):
        for k, V in sched:
            if k == a:
                sim.set_electrodes(V)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(b - a)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms += e0.elapsed_time(e1)
    t_region1 = time.time()
    st1 = sim.stats()
    o = sim.observe()
    iters = (st1["poisson_iters"] - st0["poisson_iters"]) / steps
    sb, sp = STEP_BYTES[w.dim]
    gbs = w.sites * (sb + sp * iters) / (ms / 1e3 / steps) / 1e9
    out = {"workload": name, "sites": w.sites, "value": w.sites * steps / (ms / 1e3) / 1e6,
           "unit": UNIT, "lb_steps_timed": steps, "timed_from_step": t,
           "electrode_switches_timed": len(cuts), "ms_per_lb_step": ms / steps,
           "poisson_iters_per_lb_step": iters, "step_gbs_model": gbs,
           "step_model_frac": gbs / peak, "peak_source": peak_kind,
           "collide_variant": VARIANT_NAMES.get(variant, str(variant)),
           "status": o["status"], "mass_drift": float(np.abs(o["mass"] / m0 - 1).max()),
           "window": (t_region0, t_region1)}
    sim.close()
    return out


def run_batched(args, dev, plain_mlups, peak, peak_kind, clk):
    """The 64-instance sweep (uneven 3D lattices from 48^3 to 128x64x64, viscosity ratio,
    contact angle and electrode potential drawn per instance) as one batch: per-instance
    collide kernels from the autotuner, one graph launch per coupled step for all
    instances. Same timing rules as the plain arm (device events, inputs resident).

    Two windows of --batched-steps x --batched-lb-steps steps. The early one follows the
    warm-up (a few hundred steps into the runs, where the charge is still relaxing and the
    Gauss-law solves iterate most steps). The headline one is taken once every instance has
    run --batched-settle-steps steps: the plain arm is timed thousands of steps into its run,
    and the solves' CG iterations per step only settle after ~3000 steps, so this window
    compares the two forms in the same state of the runs."""
    import collections
    import torch
    from paper_2608_12868_b300 import lbehd
    from paper_2608_12868_b300 import workloads as W
    ws = W.batched_sweep(n=args.batched)
    stream = torch.cuda.Stream(dev)
    t0 = time.perf_counter()
    batch = lbehd.Batch(ws, stream=stream, device=dev.index)
    batch.step(1)
    variants, _ = batch.autotune(reps=10)
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t0
    L = args.batched_lb_steps
    steps = max(1, args.batched_steps)
    sites = sum(w.sites for w in ws)
    sb, sp = STEP_BYTES[3]

    def window():
        st0 = batch.stats()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_region0 = time.time()
        ev0.record(stream)
        for _ in range(steps):
            batch.step(L)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        t_region1 = time.time()
        ms = ev0.elapsed_time(ev1)
        st1 = batch.stats()
        iters = (st1["poisson_iters"] - st0["poisson_iters"]) / (L * steps * len(ws))
        gbs = sites * (sb + sp * iters) / (ms / 1e3 / (L * steps)) / 1e9
        return {"lb_steps_before": st0["steps"], "ms": ms,
                "value": sites * L * steps / (ms / 1e3) / 1e6, "iters": iters, "gbs": gbs,
                "gpu_launches": st1["kernels"] - st0["kernels"],
                "graph_launches": st1["graph_launches"] - st0["graph_launches"],
                "window": (t_region0, t_region1)}

    for _ in range(args.warmup):
        batch.step(L)
    torch.cuda.synchronize(dev)
    t_w = time.perf_counter()
    while time.perf_counter() - t_w < args.warmup_seconds:
        batch.step(L)
        torch.cuda.synchronize(dev)
    early = window()
    while batch.stats()["steps"] < args.batched_settle_steps:
        batch.step(L)
    torch.cuda.synchronize(dev)
    m0 = [o["mass"] for o in batch.observe()]
    main = window()
    obs = batch.observe()
    drift = max(float(np.abs(o["mass"] / m - 1).max()) for o, m in zip(obs, m0))
    out = {
        "workload": f"batched_sweep_{len(ws)}: {len(ws)} uneven 3D instances "
                    "(48^3 .. 128x64x64), one graph launch per coupled step",
        "instances": len(ws), "sites": sites, "value": main["value"], "unit": UNIT,
        "ms_per_lb_step": main["ms"] / (L * steps), "lb_steps_timed": L * steps,
        "lb_steps_before_timed": main["lb_steps_before"],
        "vs_plain": main["value"] / plain_mlups,
        "gpu_launches": main["gpu_launches"], "graph_launches": main["graph_launches"],
        "poisson_iters_per_instance_step": main["iters"],
        "step_gbs_model": main["gbs"], "step_model_frac": main["gbs"] / peak,
        "peak_source": peak_kind,
        "early_window": {"lb_steps_before_timed": early["lb_steps_before"],
                         "value": early["value"], "vs_plain": early["value"] / plain_mlups,
                         "poisson_iters_per_instance_step": early["iters"],
                         "step_model_frac": early["gbs"] / peak},
        "collide_variants": dict(collections.Counter(VARIANT_NAMES[v] for v in variants)),
        "setup_s": setup_s, "status_all_ok": all(o["status"] == 0 for o in obs),
        "mass_drift": drift, "window": main["window"],
    }
    batch.close()
    return out


def run_adjoint(args, dev):
    """The differentiable-control case (96x64x64, 16 electrodes x 20 segments of 200
    steps). Two handles from the same initial state run the same trajectory: handle A
    records a forward run and its backward pass once untimed (checkpoint allocation, graph
    capture), then is timed on a second forward + backward; handle B runs the schedule
    plainly twice, the second time timed, so that its timed steps are A's timed steps.
    CUDA events on each handle's stream."""
    import torch
    from paper_2608_12868_b300 import lbehd
    from paper_2608_12868_b300 import workloads as W
    w = W.control_3d_96x64x64()
    V = np.array([v for _, v in w.schedule])[:args.adjoint_segments]
    seg = args.adjoint_seg_steps
    T = V.shape[0] * seg

    def timed(stream, fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1), out

    sa, sb = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    A = lbehd.Simulation(w, stream=sa, device=dev.index)
    B = lbehd.Simulation(w, stream=sb, device=dev.index)
    for sim in (A, B):
        sim.step(1)
    variant, _ = A.autotune(reps=10)
    B.set_option(lbehd.OPT_COLLIDE, variant)

    def plain():
        for k in range(V.shape[0]):
            B.set_electrodes(V[k])
            B.step(seg)

    A.adjoint_forward(V, seg)
    A.adjoint_backward()
    plain()
    torch.cuda.synchronize(dev)
    t_region0 = time.time()
    it0 = B.stats()["poisson_iters"]
    plain_ms, _ = timed(sb, plain)
    plain_iters = (B.stats()["poisson_iters"] - it0) / T
    fwd_ms, L = timed(sa, lambda: A.adjoint_forward(V, seg))
    bwd_ms, g = timed(sa, A.adjoint_backward)
    t_region1 = time.time()
    info = A.adjoint_info()
    # the backward pass leaves A in the state after its forward run: B's, bit for bit
    same = all(np.array_equal(A.array(k), B.array(k)) for k in ("g", "fphi", "frho", "pot"))
    A.close()
    B.close()
    return {
        "workload": f"{w.name}: {V.shape[1]} electrodes x {V.shape[0]} segments of {seg} "
                    f"steps ({V.size} parameters), loss = final droplet x centroid",
        "steps": T, "timed_steps": f"{T + 1}..{2 * T} of the run",
        "checkpoint_every": info["checkpoint_every"], "checkpoints": info["checkpoints"],
        "potential_trajectory": bool(info["trajectory"]),
        "plain_ms_per_step": plain_ms / T, "forward_ms_per_step": fwd_ms / T,
        "backward_ms_per_step": bwd_ms / T,
        "cost_vs_plain": (fwd_ms + bwd_ms) / plain_ms,
        "backward_vs_plain": bwd_ms / plain_ms,
        "plain_poisson_iters_per_step": plain_iters,
        "adjoint_cg_iters_per_step": info["adjoint_cg_iters"] / max(info["steps_reversed"], 1),
        "same_state_as_plain": same,
        "device_gb": info["device_bytes"] / 1e9,
        "loss": L, "grad_max_abs": float(np.abs(g).max()),
        "timing": "CUDA events on each simulation's stream; same steps for plain and adjoint",
        "window": (t_region0, t_region1),
    }


def run_profile_window(args, local):
    """Warm up, then bracket --profile-steps coupled steps with cudaProfilerStart / Stop
    (for `ncu --profile-from-start off`): replayed step graphs with --poisson graph (the
    default; each step's kernels are plain graph nodes), eager launches with --poisson host.
    Prints one line, no timing. With --profile-batched N the window covers eager steps of the
    N-instance batched sweep."""
    import torch
    from paper_2608_12868_b300 import lbehd
    from paper_2608_12868_b300 import workloads as W
    torch.cuda.set_device(local)
    if args.profile_adjoint:
        # the backward pass of an adjoint run of the control case: S segments of 16 steps
        w = W.control_3d_96x64x64()
        V = np.array([v for _, v in w.schedule])[:args.profile_adjoint]
        stream = torch.cuda.Stream()
        sim = lbehd.Simulation(w, stream=stream, device=local)
        sim.step(1)
        sim.autotune(reps=5)
        sim.adjoint_forward(V, 16)
        sim.adjoint_backward()      # untimed: allocation and graph capture
        sim.adjoint_forward(V, 16)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        sim.adjoint_backward()
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"profile_window": "adjoint backward", "workload": w.name,
                          "steps": int(V.shape[0]) * 16, "info": sim.adjoint_info()}))
        return
    if args.profile_batched:
        ws = W.batched_sweep(n=args.profile_batched)
        stream = torch.cuda.Stream()
        batch = lbehd.Batch(ws, stream=stream, device=local)
        batch.step(1)
        batch.autotune(reps=5)
        batch.step(args.warmup * args.batched_lb_steps)
        batch.profile(True)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        batch.step(args.profile_steps)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"profile_window": args.profile_steps,
                          "workload": f"batched_sweep_{len(ws)}", "stats": batch.stats(),
                          "eager_class_ms": batch.profile_read()}))
        return
    w = W.WORKLOADS[args.workload]()
    stream = torch.cuda.Stream()
    mode = {"fixed": lbehd.POISSON_FIXED, "host": lbehd.POISSON_HOST,
            "graph": lbehd.POISSON_GRAPH}[args.poisson]
    sim = lbehd.Simulation(w, stream=stream, device=local, poisson_mode=mode)
    if args.collide == "tune":
        sim.step(1)
        sim.autotune(reps=20)
    else:
        sim.set_option(lbehd.OPT_COLLIDE, COLLIDE_CHOICES[args.collide])
    sim.step(args.warmup * args.lb_steps)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    sim.step(args.profile_steps)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    print(json.dumps({"profile_window": args.profile_steps, "workload": w.name,
                      "stats": sim.stats()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="droplet_3d_128x64x64")
    ap.add_argument("--lb-steps", type=int, default=200,
                    help="coupled steps per benchmark step (200: ~42 ms on 128x64x64)")
    ap.add_argument("--warmup-seconds", type=float, default=2.0)
    ap.add_argument("--collide", choices=["tune"] + list(COLLIDE_CHOICES), default="tune")
    ap.add_argument("--batched", type=int, default=64,
                    help="instances of the batched sweep measured after the plain arm (0: skip)")
    ap.add_argument("--batched-steps", type=int, default=10)
    ap.add_argument("--batched-lb-steps", type=int, default=20,
                    help="coupled steps per timed batched step (20: ~0.1 s for 64 instances)")
    ap.add_argument("--batched-settle-steps", type=int, default=4000,
                    help="coupled steps every instance runs before the batched headline window")
    ap.add_argument("--adjoint-segments", type=int, default=20,
                    help="segments of the differentiable-control schedule (0: skip the adjoint)")
    ap.add_argument("--adjoint-seg-steps", type=int, default=200)
    ap.add_argument("--other-workloads", type=int, default=1,
                    help="1: also time the 2D 128x64 run (2000 steps), the 384x128x96 "
                         "transport run (4000 steps, electrode switches) and the 128x64x64 "
                         "droplet with Table 1's densities (2000 steps); 0: skip")
    ap.add_argument("--poisson", choices=["graph", "host", "fixed"], default="graph")
    ap.add_argument("--fixed-iters", type=int, default=2)
    ap.add_argument("--check-every", type=int, default=1)
    ap.add_argument("--cpu-steps", type=int, default=8,
                    help="timed oracle steps of the cpu_baseline (after one untimed step)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="time budget of the cpu_baseline's timed oracle steps")
    ap.add_argument("--oracle-baselines", action="store_true",
                    help="only time the FP64 oracle on 1 and on all host cores (2D 128x64, "
                         "2000 steps; 3D 128x64x64, --oracle-3d-steps steps)")
    ap.add_argument("--oracle-3d-steps", type=int, default=25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="only run a profiler window of this many eager steps (for ncu)")
    ap.add_argument("--profile-adjoint", type=int, default=0,
                    help="only profile the backward pass of an adjoint run of this many "
                         "16-step segments of the control case")
    ap.add_argument("--profile-batched", type=int, default=0,
                    help="with --profile-steps: profile the batched sweep of this many instances")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)   # at least 3 untimed warm-up steps
    if args.profile_steps or args.profile_adjoint:
        run_profile_window(args, int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.oracle_baselines:
        run_oracle_baselines(args)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
