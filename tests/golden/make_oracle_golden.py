"""Writes the oracle regression fixtures oracle_regression_<case>_*.txt.

Each fixture is what the FP64 oracle computes for a small seeded problem:
the per-step records (forces, torque, pose, velocity, solid-node count) and
64 sampled populations after the last step.  They guard the oracle's
arithmetic against unintended change: a deliberate change to it rewrites
them with this script, and its commit names the passage of the paper that
justifies it.  Only the oracle and the seeded input generators are called.

    python tests/golden/make_oracle_golden.py
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402

HISTORY_FIELDS = ("t", "fx", "fy", "torque", "fpen_x", "fpen_y", "tpen", "x", "y", "theta",
                  "vx", "vy", "omega", "n_solid")
NSAMPLE = 64


def _imposed_disk_mixed():
    p = wl.mixed_bc_box(30, 18, seed=5, west="velocity", east="zerograd", south="noslip", north="velocity",
                        tau=0.62, body={"radius": 4.2, "x": 12.3, "y": 8.6, "motion": "imposed", "axis": 1,
                                        "amp": 1.5, "freq": 0.02, "phase": 0.4, "u_ref": 0.05, "d_ref": 8.4})
    p["init"] = {"rho": 1.0, "u": (0.02, 0.0)}
    return p, None, 40


def _free_disk_periodic():
    r = 3.6
    m = 2.0 * math.pi * r * r
    p = wl.periodic_box(24, 20, tau=0.7, g_fluid=(2e-5, 0.0),
                        body={"radius": r, "x": 11.4, "y": 9.7, "vx": 0.003, "vy": -0.002, "omega": 0.001,
                              "motion": "free", "mass": m, "inertia": 0.5 * m * r * r, "dof_mask": 7,
                              "stiff": (1e-3, 2e-3, 0.0), "damp": (1e-3, 0.0, 0.0), "q0": (11.4, 9.7, 0.0),
                              "f_ext": (2e-4, 0.0, 0.0),
                              "u_ref": 0.05, "d_ref": 2 * r})
    return p, wl.random_populations(24, 20, seed=31, amp=0.02, u_amp=0.03), 40


def _paper_channel():
    # Sec. 3.1's boundaries: velocity inlet, convective outlet, symmetry walls
    p = wl.mixed_bc_box(32, 14, seed=6, west="velocity", east="convective", south="symmetry", north="symmetry",
                        tau=0.56, body={"radius": 3.0, "x": 10.2, "y": 7.1, "motion": "imposed", "axis": 1,
                                        "amp": 0.75, "freq": 0.01, "phase": math.pi / 2, "u_ref": 0.048,
                                        "d_ref": 6.0})
    p["bc"]["west"] = {"kind": "velocity", "u": (0.048, 0.0)}
    p["bc"]["east"] = {"kind": "convective", "u": (0.048, 0.0)}
    p["init"] = {"rho": 1.0, "u": (0.048, 0.0)}
    return p, None, 40


def _ellipse_bgk():
    p = wl.mixed_bc_box(26, 16, seed=7, west="velocity", east="zerograd", south="noslip", north="noslip",
                        tau=0.66, body={"shape": "ellipse", "radius": 4.5, "radius_b": 2.0, "x": 12.6, "y": 8.2,
                                        "theta": 0.3, "motion": "imposed", "axis": 2, "amp": 0.3, "freq": 0.02,
                                        "u_ref": 0.04, "d_ref": 4.0})
    p["collision"] = "bgk"
    p["init"] = {"rho": 1.0, "u": (0.03, 0.0)}
    return p, None, 30


CASES = {
    "imposed_disk_mixed_30x18": _imposed_disk_mixed,
    "free_disk_periodic_24x20": _free_disk_periodic,
    "paper_channel_32x14": _paper_channel,
    "ellipse_bgk_26x16": _ellipse_bgk,
}


def run_case(name):
    """(history rows, sample indices [a, j, i], sampled populations)."""
    p, f0, steps = CASES[name]()
    sim = oracle.OracleSim(p, hist_cap=steps + 8)
    if f0 is not None:
        sim.set_populations(f0)
    else:
        ini = p.get("init", {})
        u = ini.get("u", (0.0, 0.0))
        shape = (p["ny"], p["nx"])
        sim.init_equilibrium(np.full(shape, ini.get("rho", 1.0)), np.full(shape, u[0]), np.full(shape, u[1]))
    sim.step(steps)
    h = sim.history(0, steps)
    cols = [oracle.RECORD_FIELDS.index(k) for k in HISTORY_FIELDS]
    f = sim.populations()
    rng = np.random.default_rng(sum(map(ord, name)))
    idx = np.stack([rng.integers(0, 9, NSAMPLE), rng.integers(0, p["ny"], NSAMPLE),
                    rng.integers(0, p["nx"], NSAMPLE)], axis=1)
    return h[:, cols], idx, f[idx[:, 0], idx[:, 1], idx[:, 2]]


def paths(name):
    return (os.path.join(HERE, f"oracle_regression_{name}_history.txt"),
            os.path.join(HERE, f"oracle_regression_{name}_populations.txt"))


def main():
    for name in CASES:
        hist, idx, vals = run_case(name)
        ph, pp = paths(name)
        head = (f"FP64 oracle, case {name} (tests/golden/make_oracle_golden.py); "
                "one row per step; columns: " + " ".join(HISTORY_FIELDS))
        np.savetxt(ph, hist, fmt="%.17g", header=head)
        head = (f"FP64 oracle, case {name} (tests/golden/make_oracle_golden.py); "
                "populations after the last step; columns: a j i f")
        np.savetxt(pp, np.column_stack([idx, vals]), fmt=["%d", "%d", "%d", "%.17g"], header=head)
        print(name, hist.shape, flush=True)


if __name__ == "__main__":
    main()
