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
import contextlib
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
LEGS = ("f64", "f16", "adjoint", "batched", "sedimenting", "paper", "several")   # comparison legs after the headline
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
    if launch[0] == "pair":
        return f"vp_mrt_step_pair<{PREC_ID[prec]}, 5, 0>"
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
    "vp_mrt_step_pair<": ("vplbm_internal.cuh", "vplbm_node.cuh", "step_scalar.cuh", "step_pair.cuh", "step_pair.cu"),
    "vp_mrt_sweep<": ("vplbm_internal.cuh", "vplbm_node.cuh", "step_scalar.cuh", "step_pair.cuh", "sweep.cu"),
}


_C_COMMENT = re.compile(rb"//[^\n]*|/\*.*?\*/", re.S)
_SPACE = re.compile(rb"\s+")


def kernel_source_hash(kernel: str = "vp_mrt_step<") -> str:
    """Hash of the code of one step kernel's sources, comments left out and
    white space collapsed: a change to the code invalidates the kernel's
    counters, a change to a comment or to the layout does not."""
    files = next(v for k, v in KERNEL_SOURCES.items() if kernel.startswith(k))
    h = hashlib.sha256()
    paths = [os.path.join(ROOT, "include", "vplbm.h")] + [os.path.join(CSRC, f) for f in files]
    for path in paths:
        with open(path, "rb") as fh:
            h.update(os.path.basename(path).encode())
            h.update(_SPACE.sub(b" ", _C_COMMENT.sub(b" ", fh.read())).strip())
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


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cut_rows(p: dict, lo: int, hi: int) -> dict:
    """Rows [lo, hi) of the workload as a lattice of their own: no-slip walls
    at the cut edges (a south or north wall of the workload stays where the
    rows reach it, unless it is periodic), the west and east walls' per-row
    velocity profiles cut to the same rows, and the bodies whose centre lies
    in the rows kept at the same place relative to them (the others left
    out)."""
    wall = {"kind": "noslip", "u": (0.0, 0.0)}
    whole = lo == 0 and hi == p["ny"]

    def edge(side, reached):
        keep = whole or (reached and p["bc"][side]["kind"] != "periodic")
        return p["bc"][side] if keep else wall

    bc = dict(p["bc"], south=edge("south", lo == 0), north=edge("north", hi == p["ny"]))
    for side in ("west", "east"):
        d = dict(bc[side])
        for key in ("ux_profile", "uy_profile"):
            if d.get(key) is not None:
                d[key] = np.asarray(d[key], dtype=np.float64)[lo:hi].copy()
        bc[side] = d
    q = dict(p, ny=hi - lo, bc=bc)
    b = p.get("body")
    q["body"] = dict(b, y=b["y"] - lo) if b is not None and lo <= b["y"] < hi else None
    if p.get("bodies"):
        q["bodies"] = [dict(c, y=c["y"] - lo) for c in p["bodies"] if lo <= c["y"] < hi]
    return q


def strip_problems(p: dict, n: int) -> list:
    """The workload cut into n disjoint full-width strips of rows, each an
    independent lattice (`cut_rows`)."""
    ny = p["ny"]
    bounds = [round(k * ny / n) for k in range(n + 1)]
    return [cut_rows(p, bounds[k], bounds[k + 1]) for k in range(n)]


def row_band(p: dict, rows: int) -> dict:
    """`rows` full-width rows of the workload centred on its body (the
    middle rows without one), as a lattice of their own (`cut_rows`)."""
    b = p.get("body")
    yc = b["y"] if b is not None else p["ny"] / 2
    lo = int(min(max(0, round(yc - rows / 2)), p["ny"] - rows))
    return cut_rows(p, lo, lo + rows)


def _oracle_strip(args):
    """One host process: `warmup` untimed then `steps` timed FP64 oracle
    steps of one strip; returns (node updates timed, seconds)."""
    q, warmup, steps = args
    import oracle
    sim = oracle.OracleSim(q, hist_cap=16)
    u = q["init"]["u"]
    shape = (q["ny"], q["nx"])
    sim.init_equilibrium(np.ones(shape), np.full(shape, u[0]), np.full(shape, u[1]))
    sim.step(warmup)
    t0 = time.perf_counter()
    sim.step(steps)
    return q["nx"] * q["ny"] * steps, time.perf_counter() - t0


def oracle_all_cores(p: dict, warmup: int, steps: int, cores: int):
    """The oracle as it stands (single-threaded C) in one spawned process per
    host core, each on its own strip of the workload: node updates of all
    strips over the slowest strip's time (MLUPS)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_strip, [(q, warmup, steps) for q in strip_problems(p, cores)])
    return sum(r[0] for r in res) / max(r[1] for r in res) / 1e6


def cpu_baseline(problem: dict, budget_s: float = 10.0):
    """The FP64 oracle on the host cores: one thread on time steps of the
    full lattice, and one process per core on the lattice cut into strips."""
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
    one_core = nodes * steps / dt / 1e6
    cores = host_cores()
    # as many steps of the full lattice (in strips) as one core would do in
    # about budget_s seconds on its strip
    strip_steps = max(2, int(budget_s * one_core * 1e6 * cores / nodes))
    all_cores = oracle_all_cores(problem, 1, strip_steps, cores)
    return {"value": all_cores, "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1core": one_core, "value_allcores": all_cores,
            "sample": f"all cores: {strip_steps} FP64 time steps of the full {problem['nx']}x{problem['ny']} lattice "
                      f"cut into {cores} full-width strips, one single-threaded oracle process per core, "
                      f"after 1 untimed step (node updates of all strips over the slowest strip's time); "
                      f"one core: {steps} step{'s' if steps != 1 else ''} of the whole lattice after 1 untimed"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    p = workload(args.workload)
    cores = host_cores()
    nodes = p["nx"] * p["ny"]
    # Each step a bounded sample of the workload: when W + K oracle steps of
    # the whole lattice would take more than about a minute on the host
    # cores, every step runs on a band of rows through the body (the same
    # width, boundary rules and body; no-slip walls at the cut edges) just
    # large enough for the run to end in about a minute.  The rate is per
    # node update, so the band only sets how long the run takes.
    budget_s = 60.0
    t0 = time.perf_counter()
    oracle_all_cores(p, 0, 1, cores)
    one_step = time.perf_counter() - t0
    frac = min(1.0, budget_s / ((args.warmup + args.steps) * one_step))
    q = p
    if frac < 1.0:
        rows = max(4 * cores, int(round(frac * p["ny"])))
        q = row_band(p, rows)
    value = oracle_all_cores(q, args.warmup, args.steps, cores)
    desc = (f"{args.steps} FP64 oracle time steps (after {args.warmup} untimed) of "
            + (f"the full {p['nx']}x{p['ny']} lattice" if q is p else
               f"a {q['nx']}x{q['ny']} band of the {p['nx']}x{p['ny']} lattice through the body")
            + f" cut into {cores} full-width strips, one single-threaded oracle process per host core; "
            f"node updates of all strips over the slowest strip's time")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": nodes / (value * 1e6) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(p, args.precision, world),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
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
                s2.autotune(20)
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
        # the gradient before the sweep: the sweep's 50 000 steps keep the
        # GPU at high power for about half a minute
        if "adjoint" in legs:
            compare["adjoint"] = run_adjoint(args, torch, compare.get("f64"))
        if "batched" in legs:
            compare["batched"] = run_batched(args, torch, stream)
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
    """The 64-member spring-mounted sweep (uneven lattices, reduced velocity
    in [3, 12], m/(rho pi R^2) = 10; --sweep-members N keeps its N smallest,
    for profiling): the three batch modes timed over the same 2 000 steps, the full 50 000-step run on the autotuned mode with the
    response of every member (A*, omega*, k*_eff of Sec. 3.3 over the second
    half), the FP64 plain path (one member after another) over 2 000 steps,
    and the FP32 records of the smallest, a median and the largest member
    against their FP64 runs."""
    import paper_1905_05110_gb300 as vp
    from paper_1905_05110_gb300.viv import viv_response
    probs = wl.viv_sweep()
    if args.sweep_members:
        probs = sorted(probs, key=lambda q: q["nx"] * q["ny"])[:args.sweep_members]
    steps = args.sweep_steps or probs[0]["steps"]
    nodes = sum(p["nx"] * p["ny"] for p in probs)
    peak, _ = measured_peak()
    k_cmp = min(2000, steps)
    b = vp.Batch(probs, precision="f32", history_capacity=steps + 64, stream=stream)
    b.init_from_problems()
    tuned = b.autotune(32)
    modes = {}
    for mode in ("branches", "tiles", "persistent"):
        b.set_mode(mode)
        b.init_from_problems()
        b.step(64)
        b.sync()
        t = time_device(b, k_cmp, stream, torch)
        b.sync()
        gbs = 72 * nodes * k_cmp / t / 1e9
        modes[mode] = {"mlups": nodes * k_cmp / t / 1e6, "steps": k_cmp, "gbs_algorithmic": gbs,
                       "frac_of_hbm": gbs / peak,
                       "launch": (list(b.launch()[:3]) if mode == "tiles" else
                                  list(b.persistent()[:5]) if mode == "persistent" else list(b.members[0].launch()))}
    b.set_mode(tuned[0])
    b.init_from_problems()
    b.sync()
    t = time_device(b, steps, stream, torch)
    b.sync()
    mlups = nodes * steps / t / 1e6
    half = steps // 2
    rows = []
    hists = []
    for p, m in zip(probs, b.members):
        h = m.history(0, steps)
        hists.append(h)
        body = p["body"]
        u_star = body["u_ref"] / (math.sqrt(body["stiff"][1] / body["mass"]) / (2 * math.pi) * body["d_ref"])
        r = viv_response(h[half:, 7], body["q0"][1], body["d_ref"], body["u_ref"], body["mass"],
                         body["stiff"][1])
        rows.append({"lattice": f"{p['nx']}x{p['ny']}", "u_star": round(u_star, 6), **r,
                     "mean_cd": float(h[half:, 4].mean()), "rms_cl": float(np.sqrt((h[half:, 5] ** 2).mean()))})
    # FP64 plain path: every member on its own over the same 2 000 steps
    t64 = 0.0
    for p in probs:
        s64 = vp.Simulation(p, precision="f64", history_capacity=64, stream=stream)
        s64.init_from_problem()
        s64.step(2)
        s64.sync()
        t64 += time_device(s64, k_cmp, stream, torch)
        s64.close()
    mlups64 = nodes * k_cmp / t64 / 1e6
    # accuracy: FP32 batched records against FP64 runs of the same members
    acc_steps = min(3000, steps)
    order = sorted(range(len(probs)), key=lambda k: probs[k]["nx"] * probs[k]["ny"])
    acc = {}
    for label, k in (("smallest", order[0]), ("median", order[len(order) // 2]), ("largest", order[-1])):
        s64 = vp.Simulation(probs[k], precision="f64", history_capacity=acc_steps, stream=stream)
        s64.init_from_problem()
        s64.step(acc_steps)
        h64 = s64.history(0, acc_steps)
        s64.close()
        h32 = hists[k][:acc_steps]
        hh = acc_steps // 2
        acc[label] = {"member": k, "lattice": f"{probs[k]['nx']}x{probs[k]['ny']}",
                      "max_abs_dcl": float(np.max(np.abs(h32[:, 5] - h64[:, 5]))),
                      "max_abs_dcd": float(np.max(np.abs(h32[:, 4] - h64[:, 4]))),
                      "p99_abs_dcl": float(np.percentile(np.abs(h32[:, 5] - h64[:, 5]), 99)),
                      "p99_abs_dcd": float(np.percentile(np.abs(h32[:, 4] - h64[:, 4]), 99)),
                      "steps_solid_count_differs": int(np.sum(h32[:, 15] != h64[:, 15])),
                      "max_abs_dy_over_d": float(np.max(np.abs(h32[:, 7] - h64[:, 7])) / probs[k]["body"]["d_ref"]),
                      "mean_cd_rel_diff_2nd_half": float(abs(h32[hh:, 4].mean() - h64[hh:, 4].mean())
                                                         / abs(h64[hh:, 4].mean()))}
    b.close()
    gbs = 72 * nodes * steps / t / 1e9
    return {"members": len(probs), "nodes": nodes, "steps": steps, "mode": tuned[0], "launch": list(tuned),
            "mlups": mlups, "gbs_algorithmic": gbs, "frac_of_hbm": gbs / peak, "seconds": t,
            "modes_2000_steps": modes,
            "f64_plain_sequential_mlups": mlups64, "f64_plain_steps": k_cmp,
            "speedup_vs_f64_plain": mlups / mlups64,
            "accuracy_vs_f64_3000_steps": acc,
            "response_window": [half, steps],
            "response": rows,
            "paper_context_k_eff": {"note": "Sec. 3.3 (D = 41, U0 = 0.0488, another lattice): context only",
                                    "k_star": [9, 19, 28], "k_eff_star": [0.058, 3.20, 16.37]}}


def _objective_f64(p, nsteps, w0, stream, torch):
    """J = mean C_D + RMS C_L over [w0, nsteps) of an FP64 forward run, and
    the run's CUDA-event time."""
    import paper_1905_05110_gb300 as vp
    g = vp.Simulation(p, precision="f64", history_capacity=nsteps + 8, stream=stream)
    g.init_from_problem()
    t = time_device(g, nsteps, stream, torch)
    h = g.history(0, nsteps)
    g.close()
    return float(h[w0:, 4].mean() + np.sqrt(np.mean(h[w0:, 5] ** 2))), t


def run_adjoint(args, torch, f64_compare):
    """The gradient workload as specified: 1024 x 512 imposed-oscillation
    disk, 20 000 steps, checkpoints every 141 steps; gradient of
    J = mean C_D + RMS C_L over the second half w.r.t. the 512-entry inlet
    profile, eta, s_nu and s_e (515 values), by the FP32 discrete adjoint
    (the timed product path) and the FP64 one, each checked against central
    finite differences of FP64 forward runs on the GPU along 8 seeded random
    unit directions, h = 1e-4 of each parameter's scale."""
    import paper_1905_05110_gb300 as vp
    p = wl.adjoint_disk()
    nsteps, ck = p["steps"], p["checkpoint_interval"]
    if args.adjoint_steps and args.adjoint_steps != nsteps:   # a shorter run: checkpoints every sqrt(N)
        nsteps, ck = args.adjoint_steps, max(1, int(round(args.adjoint_steps ** 0.5)))
    w0 = nsteps // 2
    nodes = p["nx"] * p["ny"]
    nparams = p["ny"] + 3
    stream = torch.cuda.current_stream()
    peak, _ = measured_peak()
    grads, js, secs = {}, {}, {}
    for prec in ("f32", "f64"):
        sim = vp.Simulation(p, precision=prec, history_capacity=nsteps + 8, stream=stream)
        sim.init_from_problem()
        if prec == "f32":
            launch = sim.autotune(8)   # the forward and recomputed steps use the tuned step kernel
        # FP32: one untimed call, then the median of three, each from the
        # initial state (a call leaves the context at the state after its
        # forward run); the FP64 call, about 10 s, once
        reps = 3 if prec == "f32" else 1
        if prec == "f32":
            sim.adjoint(nsteps, w0, 1.0, 1.0, checkpoint_interval=ck)
        tt = []
        with (ClockSampler(torch.cuda.current_device()) if prec == "f32" else contextlib.nullcontext()) as cs:
            for _ in range(reps):
                if prec == "f32":
                    sim.init_from_problem()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                grads[prec], js[prec] = sim.adjoint(nsteps, w0, 1.0, 1.0, checkpoint_interval=ck)
                tt.append(time.perf_counter() - t0)
        secs[prec] = float(np.median(tt))
        if prec == "f32":
            secs_f32_all = [round(t, 4) for t in tt]
            clocks_f32 = cs.summary()
            sim.init_from_problem()
            t_fwd32 = time_device(sim, nsteps, stream, torch)
        sim.close()
    # central differences of FP64 forward runs
    prof = p["bc"]["west"]["ux_profile"]
    scale = np.concatenate([np.full(p["ny"], 0.04), [p["eta"], p["s"][7], p["s"][1]]])
    rng = np.random.default_rng(2024)
    h = 1e-4
    rows, t_runs = [], []
    for _ in range(8):
        v = rng.standard_normal(nparams)
        v /= np.linalg.norm(v)
        dth = h * scale * v
        jpm = []
        for sign in (1.0, -1.0):
            q = wl.with_params(p, u_in_profile=prof + sign * dth[:-3], eta=p["eta"] + sign * dth[-3],
                               s_nu=p["s"][7] + sign * dth[-2], s_e=p["s"][1] + sign * dth[-1])
            jv, tr = _objective_f64(q, nsteps, w0, stream, torch)
            jpm.append(jv)
            t_runs.append(tr)
        fd = (jpm[0] - jpm[1]) / (2 * h)
        a64 = float(grads["f64"] @ (scale * v))
        a32 = float(grads["f32"] @ (scale * v))
        rows.append({"fd": fd, "adjoint_f64": a64, "adjoint_f32": a32,
                     "rel_diff_f64": abs(a64 - fd) / abs(fd), "rel_diff_f32": abs(a32 - fd) / abs(fd)})
    t_fwd64 = float(np.mean(t_runs))
    gbs = 216 * nodes * nsteps / secs["f32"] / 1e9
    return {"lattice": f"{p['nx']}x{p['ny']}", "steps": nsteps, "window": [w0, nsteps], "checkpoint_interval": ck,
            "params": nparams, "launch": list(launch),
            "seconds": secs["f32"], "seconds_f32_repeats": secs_f32_all, "clocks_f32": clocks_f32,
            "seconds_f64_adjoint": secs["f64"], "J": js["f32"], "J_f64": js["f64"],
            "grad_norm": float(np.linalg.norm(grads["f32"])),
            "grad_rel_diff_f32_vs_f64": float(np.linalg.norm(grads["f32"] - grads["f64"]) /
                                              np.linalg.norm(grads["f64"])),
            "gbs_at_216_bytes_per_node_step": gbs, "frac_of_hbm": gbs / peak,
            # every phase of the call: the forward run with its checkpoints
            # (72 B per node-step), the recomputation (72) and the reverse
            # kernel (pulled state and incoming adjoint read, outgoing adjoint
            # written: 108)
            "gbs_all_phases_252_bytes_per_node_step": 252 * nodes * nsteps / secs["f32"] / 1e9,
            "frac_of_hbm_all_phases": 252 * nodes * nsteps / secs["f32"] / 1e9 / peak,
            "forward_f32_seconds": t_fwd32, "forward_f64_seconds_measured": t_fwd64,
            "speedup_vs_fd_f64": 2 * nparams * t_fwd64 / secs["f32"],
            "speedup_vs_fd_f64_how": "2 x 515 FP64 forward runs at the mean CUDA-event time of the 16 FD runs "
                                     "measured here, over the FP32 adjoint's wall time",
            "speedup_vs_fd_f32_forward": 2 * nparams * t_fwd32 / secs["f32"],
            "fd_check": {"directions": 8, "h_relative": h, "seed": 2024,
                         "max_rel_diff_f64": max(r["rel_diff_f64"] for r in rows),
                         "max_rel_diff_f32": max(r["rel_diff_f32"] for r in rows), "rows": rows}}


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
    ap.add_argument("--adjoint-steps", type=int, default=0,
                    help="steps of the gradient leg (default: the workload's 20 000, checkpoints every 141)")
    ap.add_argument("--sweep-steps", type=int, default=0,
                    help="steps of the sweep leg's full run (default: the workload's 50 000)")
    ap.add_argument("--sweep-members", type=int, default=0,
                    help="the sweep leg on its N smallest members only (default: all 64; for profiling)")
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
