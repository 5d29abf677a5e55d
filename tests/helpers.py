"""Helpers shared by the GPU parity tests (no test functions here)."""
import numpy as np

import oracle
import workloads as wl

REC = {n: k for k, n in enumerate(oracle.RECORD_FIELDS)}


def rel_err(a, b) -> float:
    """max |a - b| / max |b| (scale-normalised, per field)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b))
    if scale == 0:
        return float(np.max(np.abs(a)))
    return float(np.max(np.abs(a - b)) / scale)


def dev_err(a, b, rho0=1.0) -> float:
    """Error of populations relative to the size of their deviation from rest."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None] * rho0
    return rel_err(np.asarray(a) - w, np.asarray(b) - w)


def make_pair(problem, precision, hist_cap=4096, init="problem", f0=None):
    import paper_1905_05110_gb300 as vp
    gpu = vp.Simulation(problem, precision=precision, history_capacity=hist_cap)
    orc = oracle.OracleSim(problem, hist_cap=hist_cap)
    if f0 is not None:
        gpu.set_populations(f0)
        orc.set_populations(f0)
    elif init == "problem":
        gpu.init_from_problem()
        ini = problem.get("init", {})
        u = ini.get("u", (0.0, 0.0))
        shape = (problem["ny"], problem["nx"])
        orc.init_equilibrium(np.full(shape, ini.get("rho", 1.0)), np.full(shape, u[0]),
                             np.full(shape, u[1]))
    return gpu, orc


def moving_bodies(nx, ny):
    """One body of each motion kind, placed in an nx x ny box."""
    r = min(nx, ny) / 6.0
    return {
        "fixed": {"radius": r, "x": nx * 0.41, "y": ny * 0.52, "motion": "fixed",
                  "u_ref": 0.05, "d_ref": 2 * r},
        "imposed": {"radius": r, "x": nx * 0.43, "y": ny * 0.47, "motion": "imposed", "axis": 1,
                    "amp": 0.2 * r, "freq": 0.01, "phase": 0.3, "u_ref": 0.05, "d_ref": 2 * r},
        "free": {"radius": r, "x": nx * 0.47, "y": ny * 0.49, "vx": 0.004, "vy": -0.003,
                 "omega": 0.001, "motion": "free", "mass": 2.0 * np.pi * r * r,
                 "inertia": np.pi * r ** 4, "stiff": (0.0, 1e-3, 0.0), "q0": (0.0, ny * 0.5, 0.0),
                 "damp": (0.01, 0.0, 0.0), "f_ext": (0.0, -1e-4, 0.0), "dof_mask": 7,
                 "u_ref": 0.05, "d_ref": 2 * r},
    }
