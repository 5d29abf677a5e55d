"""Benchmark of the VP-LBM hot path: MLUPS and fraction of the HBM roofline.

One bench step is one time step (Algorithm 1: stream, collide with
penalization, force/torque reduction, body update) over the whole lattice of
the imposed-oscillation workload (2048 x 1024 D2Q9, disk D = 40, FP32
deviation storage).  The device-timed value has the populations resident in
HBM; the e2e value goes through the C ABI with host buffers (initial fields
uploaded from pinned memory, force history and final fields read back).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica (the single-lattice
path has no exchange step): value = node updates of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = "D2Q9 VP-MRT MLUPS & % HBM roofline; FP32/batched/adjoint vs FP64 plain, same GPU"
UNIT = "MLUPS"
BYTES_PER_NODE = {"f64": 144, "f32": 72, "f16": 36}   # 9 loads + 9 stores of one population
PREC_ID = {"f64": 0, "f32": 1, "f16": 2}
LEGS = ("f64", "f16", "batched", "adjoint", "sedimenting", "paper", "several")   # comparison legs after the headline
FALLBACK_HBM_GBS = 6800.0
REPEATS = 5   # timed regions of K steps; the line reports the median
PROFILE_DIR = os.path.join(ROOT, "profiles")
CSRC = os.path.join(ROOT, "paper_1905_05110_gb300", "csrc")


def dominant_kernel(prec: str, launch, kinds: dict) -> str:
    """The step kernel that made most of the node updates of a timed region,
    from the launches of each kind made inside it (MRT collision, disk)."""
    work = {"two_step": 2 * kinds.get("two_step", 0), "one_step": kinds.get("one_step", 0),
            "tma": kinds.get("tma", 0)}
    top = max(work, key=work.get)
    if top == "two_step":
        return f"vp_mrt_step2<{PREC_ID[prec]}, 0, 0>"
    if top == "tma":
        return f"vp_mrt_step_tma<{PREC_ID[prec]}>"
    # single steps of a two-step choice run the 40-register kernel
    minb = {"scalar": 4, "scalar48": 5, "scalar40": 6, "fused2": 6, "tma": 6}[launch[0]]
    return f"vp_mrt_step<{PREC_ID[prec]}, {minb}, 0, 0>"


def workload(name: str) -> dict:
    if name == "oscillating_2048x1024":
        return wl.oscillating_disk()
    if name == "sedimenting_1024x4096":
        return wl.sedimenting_disk()
    if name == "paper_cylinder_1230x410":
        return wl.paper_oscillating_cylinder()
    if name == "channel_256x128":
        return wl.channel_fixed_disk()
    if name == "several_bodies_2048x1024":
        return wl.several_bodies()
    raise SystemExit(f"unknown workload {name}")


def bench_config(p: dict, prec: str, world: int) -> dict:
    """The workload's config, the same on both arms of the comparison."""
    pop_mb = p["nx"] * p["ny"] * BYTES_PER_NODE[prec] / 1e6   # read + written per step
    return {"workload": p["name"], "nx": p["nx"], "ny": p["ny"],
            "storage": {"f32": "f32 deviation", "f16": "f16 deviation", "f64": "f64"}[prec],
            "parallelism": f"replicas x{world}",
            "l2": f"not flushed: populations {pop_mb:.0f} MB read+write per step > 129 MB L2"
                  if pop_mb > 129 else f"not flushed: populations {pop_mb:.0f} MB per step fit the 129 MB L2"}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# Sources that make up each step kernel's code: the public header, the
# internal headers and the translation unit that instantiates it.
KERNEL_SOURCES = {
    "vp_mrt_step<": ("vplbm_internal.cuh", "vplbm_node.cuh", "step_scalar.cuh", "step_kernels.cu"),
    "vp_mrt_step2<": ("vplbm_internal.cuh", "vplbm_node.cuh", "step_fused2.cu"),
    "vp_mrt_step_tma<": ("vplbm_internal.cuh", "vplbm_node.cuh", "step_tma.cu"),
}


def kernel_source_hash(kernel: str = "vp_mrt_step<") -> str:
    """Hash of the sources of one step kernel (any change to them invalidates
    its counters)."""
    files = next(v for k, v in KERNEL_SOURCES.items() if kernel.startswith(k))
    h = hashlib.sha256()
    paths = [os.path.join(ROOT, "include", "vplbm.h")] + [os.path.join(CSRC, f) for f in files]
    for path in paths:
        with open(path, "rb") as fh:
            h.update(os.path.basename(path).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if still valid."""
    stem = kernel.replace("<", "_").replace(">", "").replace(", ", "_")
    path = os.path.join(PROFILE_DIR, f"{stem}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.e+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash(kernel):
        return None
    return float(m_bytes.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
                except ValueError:
                    continue
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        loaded = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in loaded:
            for name, flag in zip(names, r[3][1:5]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(loaded),
                "power_w_max": max(r[2] for r in rows)}


def max_over_ranks(value: float, world: int, device, torch) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world <= 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def time_device(sim, steps, stream, torch):
    """CUDA-event time of `steps` time steps on the simulation's stream."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def cpu_baseline(problem: dict, budget_s: float = 12.0):
    """The FP64 oracle, single-threaded, on time steps of the same lattice."""
    import oracle
    sim = oracle.OracleSim(problem, hist_cap=64)
    u = problem["init"]["u"]
    shape = (problem["ny"], problem["nx"])
    sim.init_equilibrium(np.ones(shape), np.full(shape, u[0]), np.full(shape, u[1]))
    t0 = time.perf_counter()
    sim.step(1)
    one = time.perf_counter() - t0
    extra = max(0, min(20, int(budget_s / max(one, 1e-3)) - 1))
    t0 = time.perf_counter()
    sim.step(extra)
    dt = time.perf_counter() - t0
    steps = extra if extra > 0 else 1
    if extra == 0:
        dt = one
    nodes = problem["nx"] * problem["ny"]
    return {"value": nodes * steps / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} FP64 time steps of the full {problem['nx']}x{problem['ny']} lattice "
                      f"(after 1 untimed), plain C, one thread"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    p = workload(args.workload)
    import oracle
    nodes = p["nx"] * p["ny"]
    per_step_est = nodes * 0.5e-6
    sample = p
    if (args.steps + args.warmup) * per_step_est > 150:
        # bounded sample: a strip of the same lattice (same physics per node)
        ny = max(16, int(p["ny"] * 150 / ((args.steps + args.warmup) * per_step_est)))
        sample = dict(p, ny=ny, body=dict(p["body"], y=ny / 2.0))
    sim = oracle.OracleSim(sample, hist_cap=max(16, args.steps + args.warmup))
    u = sample["init"]["u"]
    shape = (sample["ny"], sample["nx"])
    sim.init_equilibrium(np.ones(shape), np.full(shape, u[0]), np.full(shape, u[1]))
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    value = sample["nx"] * sample["ny"] * args.steps / dt / 1e6
    desc = (f"{args.steps} FP64 oracle time steps of a {sample['nx']}x{sample['ny']} lattice "
            f"({'full workload' if sample is p else 'strip of the workload'}), one thread")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(p, args.precision, world),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1905_05110_gb300 as vp
    from paper_1905_05110_gb300 import build as vbuild

    if rank == 0 or not os.path.exists(vbuild.LIB):
        vbuild.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    p = workload(args.workload)
    nodes = p["nx"] * p["ny"]
    prec = args.precision

    sim = vp.Simulation(p, precision=prec, history_capacity=max(1024, args.steps + args.warmup + 64),
                        stream=stream)
    sim.init_from_problem()
    if args.launch:
        kern, shape = args.launch.split(":")
        bx, by = (int(v) for v in shape.split("x"))
        sim.set_launch(kern, bx, by)
    elif not args.no_autotune:
        sim.autotune(20)
    launch = sim.launch()
    sim.step(args.warmup)
    sim.sync()

    # REPEATS timed regions of exactly K steps each (device-synchronized on
    # both sides); the line reports the median one, with the launches of each
    # kernel kind made inside it
    samples = []
    with ClockSampler(local_rank) as clocks:
        for _ in range(REPEATS):
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            k0 = sim.kernel_launches()
            t = time_device(sim, args.steps, stream, torch)
            torch.cuda.synchronize()
            k1 = sim.kernel_launches()
            samples.append((max_over_ranks(t, world, dev, torch), {k: k1[k] - k0[k] for k in k1}))
    sim.sync()
    times = sorted(t for t, _ in samples)
    dt, kinds = next(s for s in samples if s[0] == times[REPEATS // 2])
    launches = sum(kinds.values())
    value = world * nodes * args.steps / dt / 1e6
    clock = clocks.summary()

    # roofline of the step kernel that did most of the region's node updates
    # (a two-step launch does the work, and the algorithmic bytes, of two
    # steps; the one-thread lookahead launches move no lattice bytes)
    peak, peak_kind = measured_peak()
    kname = dominant_kernel(prec, launch, kinds)
    steps_per_launch = 2 if kname.startswith("vp_mrt_step2<") else 1
    algorithmic = BYTES_PER_NODE[prec] * nodes * args.steps
    achieved = algorithmic / dt / 1e9
    traffic = profiled_traffic(kname, args.workload)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                "kernel": kname, "algorithmic_bytes_per_launch": steps_per_launch * BYTES_PER_NODE[prec] * nodes,
                "launches_in_region": kinds,
                "kernel_source_sha256_16": kernel_source_hash(kname)}
    repeats = {"n": REPEATS, "ms_per_step": [t / args.steps * 1e3 for t, _ in samples],
               "median_ms_per_step": dt / args.steps * 1e3,
               "spread": (times[-1] - times[0]) / dt,
               "mlups_min_max": [world * nodes * args.steps / times[-1] / 1e6,
                                 world * nodes * args.steps / times[0] / 1e6]}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(sim, p, args.steps, torch)

    # the other precisions on the same GPU, for the FP32 / FP16 vs FP64 comparison
    compare = {}
    if not args.no_compare and rank == 0:
        for other in ("f64", "f16"):
            if other == prec or (args.legs and other not in args.legs.split(",")):
                continue
            s2 = vp.Simulation(p, precision=other, history_capacity=4096, stream=stream)
            s2.init_from_problem()
            if not args.no_autotune:
                s2.autotune(8)
            s2.step(50)
            s2.sync()
            k = max(200, min(args.steps, 2000 if other == "f64" else args.steps))
            t2 = time_device(s2, k, stream, torch)
            s2.sync()
            compare[other] = {"mlups": nodes * k / t2 / 1e6, "steps": k,
                              "gbs_algorithmic": BYTES_PER_NODE[other] * nodes * k / t2 / 1e9,
                              "launch": list(s2.launch())}
            s2.close()
        if "f64" in compare:
            compare["speedup_vs_f64"] = (nodes * args.steps / dt / 1e6) / compare["f64"]["mlups"]
        if not args.legs or "f64" in args.legs.split(","):
            compare["accuracy_vs_f64"] = run_accuracy(p, 4000, torch, stream, not args.no_autotune)

    legs = set(args.legs.split(",")) if args.legs else set(LEGS)
    if not args.no_compare and world > 1 and "batched" in legs:
        compare["batched_sharded"] = run_sharded_sweep(args, torch, stream, rank, world, dev)
    if not args.no_compare and rank == 0:
        if "batched" in legs:
            compare["batched"] = run_batched(args, torch, stream)
        if "adjoint" in legs:
            compare["adjoint"] = run_adjoint(args, torch, compare.get("f64"))
        if "sedimenting" in legs:
            compare["sedimenting_disk"] = run_other_workload("sedimenting_1024x4096", 200_000, torch, stream)
        if "paper" in legs:
            compare["paper_oscillating_cylinder"] = run_other_workload("paper_cylinder_1230x410", 40000, torch,
                                                                       stream)
        if "several" in legs:
            compare["several_bodies"] = run_other_workload("several_bodies_2048x1024", 8000, torch, stream)

    base = None
    if rank == 0 and not args.no_cpu_baseline:
        base = cpu_baseline(p)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec != "f64" else "f64",
                "data": "synthetic",
                "config": bench_config(p, prec, world), "launch": list(launch), "repeats": repeats,
                "roofline": roofline, "cpu_baseline": base, "e2e": e2e,
                "gpu_launches": launches, "clocks": clock, "compare": compare}
        print(json.dumps(line), flush=True)
    sim.close()


def run_accuracy(p, steps, torch, stream, autotune):
    """FP32 and FP16 deviation storage against FP64 storage on the same
    workload, GPU against GPU from the same initial state: C_D and C_L over
    the run, and the fields at its end."""
    import paper_1905_05110_gb300 as vp
    u0 = max(abs(p["init"]["u"][0]), abs(p["init"]["u"][1]), 1e-12)
    runs = {}
    for prec in ("f64", "f32", "f16"):
        sim = vp.Simulation(p, precision=prec, history_capacity=steps + 8, stream=stream)
        sim.init_from_problem()
        if autotune and prec != "f64":
            sim.autotune(8)
        sim.step(steps)
        sim.sync()
        runs[prec] = (sim.history(0, steps), sim.fields(), list(sim.launch()))
        sim.close()
    h64, (r64, ux64, uy64), _ = runs["f64"]
    half = steps // 2
    out = {"steps": steps, "workload": p["name"]}
    for prec in ("f32", "f16"):
        h, (r, ux, uy), launch = runs[prec]
        cd, cl = h[:, 4], h[:, 5]
        out[prec] = {
            "launch": launch,
            "max_abs_dcd": float(np.max(np.abs(cd - h64[:, 4]))),
            "max_abs_dcl": float(np.max(np.abs(cl - h64[:, 5]))),
            "mean_cd_2nd_half": float(cd[half:].mean()),
            "mean_cd_2nd_half_f64": float(h64[half:, 4].mean()),
            "rms_cl_2nd_half": float(np.sqrt((cl[half:] ** 2).mean())),
            "rms_cl_2nd_half_f64": float(np.sqrt((h64[half:, 5] ** 2).mean())),
            "max_abs_du_over_u0": float(max(np.max(np.abs(ux - ux64)), np.max(np.abs(uy - uy64))) / u0),
            "max_abs_drho": float(np.max(np.abs(r - r64))),
        }
    return out


def run_other_workload(name, steps, torch, stream):
    """FP32 rate of another workload (free body / the paper's own setup),
    with the mean C_D and RMS C_L of the second half of the run."""
    import paper_1905_05110_gb300 as vp
    p = workload(name)
    nodes = p["nx"] * p["ny"]
    sim = vp.Simulation(p, precision="f32", history_capacity=steps + 64, stream=stream)
    sim.init_from_problem()
    launch = sim.autotune(8)
    t = time_device(sim, steps, stream, torch)
    sim.sync()
    half = steps // 2
    out = {"workload": p["name"], "mlups": nodes * steps / t / 1e6, "steps": steps, "launch": list(launch)}
    bodies = p.get("bodies") or [p["body"]]
    per_body = []
    for k, b in enumerate(bodies):
        h = sim.history(0, steps, body=k)
        d = {"motion": b["motion"], "mean_cd_2nd_half": float(h[half:, 4].mean()),
             "rms_cl_2nd_half": float(np.sqrt((h[half:, 5] ** 2).mean()))}
        if b["motion"] == "free":
            d["final_pose"] = [float(v) for v in h[-1, 6:9]]
            d["final_velocity"] = [float(v) for v in h[-1, 9:12]]
            if "gravity" in p:   # settling: terminal velocity against the design value v_s = Re_t nu / D
                nu = (1.0 / p["s"][7] - 0.5) / 3.0
                vt = float(-h[-max(1, steps // 20):, 10].mean())
                d["terminal_vy_last_5pct"] = vt
                d["terminal_re"] = vt * b["d_ref"] / nu
                d["design_v_s"] = b["u_ref"]
                d["terminal_over_design"] = vt / b["u_ref"]
                d["gravity"] = p["gravity"]
                d["gravity_over_happel"] = wl.SETTLING_G_FACTOR
        per_body.append(d)
    if len(bodies) == 1:
        out.update(per_body[0])
        del out["motion"]
    else:
        out["bodies"] = per_body
    sim.close()
    return out


def run_sharded_sweep(args, torch, stream, rank, world, dev):
    """The 64-member sweep sharded over the ranks (greedy longest-processing-
    time by node count, the same partition on every rank, no exchange): the
    units all ranks processed over the slowest rank's time."""
    import paper_1905_05110_gb300 as vp
    from paper_1905_05110_gb300.sweep import member_nodes, partition_members
    probs = wl.viv_sweep()
    nodes = member_nodes(probs)
    mine = partition_members(nodes, world)[rank]
    b = vp.Batch([probs[k] for k in mine], precision="f32", history_capacity=1024, stream=stream)
    b.init_from_problems()
    b.step(64)
    b.sync()
    k = max(64, min(512, args.steps // 50))
    torch.distributed.barrier()
    torch.cuda.synchronize()
    t = time_device(b, k, stream, torch)
    b.sync()
    b.close()
    t = max_over_ranks(t, world, dev, torch)
    return {"ranks": world, "members": len(probs), "nodes": sum(nodes), "steps": k,
            "mlups": sum(nodes) * k / t / 1e6, "scaling": "strong (fixed 64-member sweep)"}


def run_batched(args, torch, stream):
    """The 64-member spring-mounted sweep (uneven lattices) in one launch per
    step, against the same members on the FP64 plain path, with the C_D / C_L
    difference of one member over a run stated."""
    import paper_1905_05110_gb300 as vp
    probs = wl.viv_sweep()
    nodes = sum(p["nx"] * p["ny"] for p in probs)
    b = vp.Batch(probs, precision="f32", history_capacity=4096, stream=stream)
    b.init_from_problems()
    shape = b.autotune(16)
    b.init_from_problems()
    b.step(64)
    b.sync()
    k = max(64, min(512, args.steps // 50))
    t = time_device(b, k, stream, torch)
    b.sync()
    mlups = nodes * k / t / 1e6
    # FP64 plain path: every member on its own, a few steps each
    t64 = 0.0
    k64 = 8
    for p in probs:
        s64 = vp.Simulation(p, precision="f64", history_capacity=64, stream=stream)
        s64.init_from_problem()
        s64.step(2)
        s64.sync()
        t64 += time_device(s64, k64, stream, torch)
        s64.close()
    mlups64 = nodes * k64 / t64 / 1e6
    # accuracy: member 0 over 3000 steps, FP32 batched vs FP64
    acc_steps = 3000
    m = b.members[0]
    b.init_from_problems()
    b.step(acc_steps)
    h32 = m.history(0, acc_steps)
    s64 = vp.Simulation(probs[0], precision="f64", history_capacity=acc_steps, stream=stream)
    s64.init_from_problem()
    s64.step(acc_steps)
    h64 = s64.history(0, acc_steps)
    s64.close()
    half = acc_steps // 2
    cd32, cd64 = h32[half:, 4].mean(), h64[half:, 4].mean()
    b.close()
    return {"members": len(probs), "nodes": nodes, "mlups": mlups, "steps": k, "launch": list(shape),
            "gbs_algorithmic": 72 * nodes * k / t / 1e9,
            "f64_plain_sequential_mlups": mlups64, "speedup_vs_f64_plain": mlups / mlups64,
            "accuracy_member0_3000_steps": {
                "lattice": f"{probs[0]['nx']}x{probs[0]['ny']}",
                "max_abs_dcl": float(np.max(np.abs(h32[:, 5] - h64[:, 5]))),
                "max_abs_dcd": float(np.max(np.abs(h32[:, 4] - h64[:, 4]))),
                "mean_cd_rel_diff_2nd_half": float(abs(cd32 - cd64) / abs(cd64))}}


def run_adjoint(args, torch, f64_compare):
    """Gradient of mean C_D + RMS C_L over the second half of 1024 x 512 runs
    w.r.t. the 512-entry inlet profile, eta, s_nu, s_e (515 values), by the
    FP32 discrete adjoint with checkpoints every 141 steps."""
    import paper_1905_05110_gb300 as vp
    p = wl.adjoint_disk()
    nsteps = min(p["steps"], max(2000, args.steps // 2))
    ck = p["checkpoint_interval"] if nsteps == p["steps"] else max(1, int(round(nsteps ** 0.5)))
    nodes = p["nx"] * p["ny"]
    sim = vp.Simulation(p, precision="f32", history_capacity=nsteps + 8)
    sim.init_from_problem()
    launch = sim.autotune(8)   # the forward and recomputed steps use the tuned step kernel
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grad, js = sim.adjoint(nsteps, nsteps // 2, 1.0, 1.0, checkpoint_interval=ck)
    dt = time.perf_counter() - t0
    sim.init_from_problem()
    t_fwd = time_device(sim, nsteps, torch.cuda.current_stream(), torch)
    sim.close()
    nparams = p["ny"] + 3
    out = {"lattice": f"{p['nx']}x{p['ny']}", "steps": nsteps, "checkpoint_interval": ck, "params": nparams,
           "seconds": dt, "forward_f32_seconds": t_fwd, "J": js, "launch": list(launch),
           "speedup_vs_fd_f32_forward": 2 * nparams * t_fwd / dt,
           "grad_norm": float(np.linalg.norm(grad))}
    if f64_compare:
        t_fd64 = 2 * nparams * nodes * nsteps / (f64_compare["mlups"] * 1e6)
        out["speedup_vs_fd_f64_plain"] = t_fd64 / dt
    return out


def run_e2e(sim, p, steps, torch):
    """Same metric through the public API with host buffers, copies timed."""
    import paper_1905_05110_gb300 as vp
    ny, nx = p["ny"], p["nx"]
    u = p["init"]["u"]
    pinned = [torch.empty((ny, nx), dtype=torch.float64, pin_memory=True) for _ in range(6)]
    pinned[0].fill_(p["init"]["rho"])
    pinned[1].fill_(u[0])
    pinned[2].fill_(u[1])
    hist = (vp.Record * steps)()
    arrs = [t.numpy() for t in pinned]

    def once():
        vp.vplbm_init_equilibrium(sim.ctx, arrs[0], arrs[1], arrs[2])
        vp.vplbm_step(sim.ctx, steps)
        lib = vp.load_library()
        st = lib.vplbm_get_history(sim.ctx, 0, steps, hist)
        if st != 0:
            raise vp.VplbmError(st, vp.vplbm_last_error())
        vp.vplbm_get_fields(sim.ctx, arrs[3], arrs[4], arrs[5])

    once()   # warm-up of the same path
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    once()
    dt = time.perf_counter() - t0
    h2d = 3 * nx * ny * 8
    d2h = 3 * nx * ny * 8 + steps * 128
    return {"value": nx * ny * steps / dt / 1e6, "unit": UNIT,
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "what": "init from pinned host fields + steps + history and fields to pinned host"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40000)
    ap.add_argument("--warmup", type=int, default=1000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="oscillating_2048x1024")
    ap.add_argument("--precision", default="f32", choices=["f32", "f16", "f64"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--launch", default="", help="fixed step kernel and block, e.g. scalar40:256x1 (no autotune)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="", help="comma-separated subset of " + ",".join(LEGS) + " (default: all)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
