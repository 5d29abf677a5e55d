"""The two-step kernel (two time steps per launch through a shared-memory
stage) against the one-step scalar kernel and the FP64 oracle.

The two-step kernel runs the one-step kernel's node arithmetic on the same
inputs, so its populations must equal the one-step kernel's bit for bit,
in FP32 and FP16 storage, over runs that mix graphs of two-step launches
with single steps.  Its force sums are reduced in another order (per-thread
float-float accumulators over the tile), so the records agree to 1e-9 of
their scale; the solid-node counts and poses (a prescribed path) exactly.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from helpers import REC, dev_err, make_pair, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library(gpu_library):
    return gpu_library


def _channel_imposed():
    return wl.oscillating_disk(nx=300, ny=130, diameter=20.0, x_c=61.3)


def _fixed_ellipse():
    p = wl.mixed_bc_box(161, 83, seed=7, west="velocity", east="zerograd", south="noslip", north="noslip", tau=0.6,
                        body={"shape": "ellipse", "radius": 14.0, "radius_b": 6.0, "x": 70.3, "y": 41.6,
                              "theta": 0.4, "motion": "fixed", "u_ref": 0.05, "d_ref": 12.0})
    p["init"] = {"rho": 1.0, "u": (0.03, 0.0)}
    return p


def _pitching_rectangle_symmetry():
    p = wl.mixed_bc_box(150, 70, seed=8, west="velocity", east="zerograd", south="symmetry", north="symmetry",
                        tau=0.62, body={"shape": "rectangle", "radius": 9.0, "radius_b": 4.0, "x": 60.2, "y": 35.3,
                                        "theta": 0.2, "motion": "imposed", "axis": 2, "amp": 0.5, "freq": 0.01,
                                        "u_ref": 0.05, "d_ref": 8.0})
    p["s"] = wl.paper_rates(0.62)
    p["bc"]["west"] = {"kind": "velocity", "u": (0.05, 0.0)}
    p["init"] = {"rho": 1.0, "u": (0.05, 0.0)}
    return p


def _periodic_random(nx, ny, body=None):
    p = wl.periodic_box(nx, ny, tau=0.7, body=body, g_fluid=(1e-5, 2e-6))
    p["f0"] = wl.random_populations(nx, ny, seed=nx + ny, amp=0.02, u_amp=0.03)
    return p


def _ragged_walls():
    # random wall-velocity profiles on every wall, moving disk, ragged size
    p = wl.mixed_bc_box(130, 37, seed=11, west="velocity", east="velocity", south="velocity", north="noslip",
                        tau=0.66, body={"radius": 6.2, "x": 40.7, "y": 18.4, "motion": "imposed", "axis": 0,
                                        "amp": 2.0, "freq": 0.02, "u_ref": 0.03, "d_ref": 12.4},
                        rates=wl.random_rates(11))
    return p


def _bgk_channel():
    p = _channel_imposed()
    p["collision"] = "bgk"
    return p


def _tiny_walls():
    # smaller than one tile in both directions, walls on every side
    p = wl.mixed_bc_box(7, 5, seed=12, west="velocity", east="zerograd", south="noslip", north="velocity", tau=0.7)
    p["init"] = {"rho": 1.0, "u": (0.02, 0.0)}
    return p


def _periodic_x_symmetry_y():
    # the mirror rule's corner nodes wrap across the periodic x edges
    p = wl.mixed_bc_box(90, 40, seed=13, west="periodic", east="periodic", south="symmetry", north="symmetry",
                        tau=0.65, body={"radius": 6.5, "x": 44.3, "y": 19.6, "motion": "imposed", "axis": 1,
                                        "amp": 2.0, "freq": 0.015})
    p["g_fluid"] = (2e-5, 0.0)
    p["f0"] = wl.random_populations(90, 40, seed=14, amp=0.02, u_amp=0.03)
    return p


def _convective_channel(nx, ny, body, u=0.048, seed=3):
    # the channel of Sec. 3.1: velocity inlet, convective outlet, symmetry walls
    p = wl.mixed_bc_box(nx, ny, seed=seed, west="velocity", east="convective", south="symmetry",
                        north="symmetry", tau=0.56, body=body)
    p["bc"]["west"] = {"kind": "velocity", "u": (u, 0.0)}
    p["bc"]["east"] = {"kind": "convective", "u": (u, 0.0)}
    p["init"] = {"rho": 1.0, "u": (u, 0.0)}
    return p


def _paper_channel_cosine():
    r = 6.0
    return _convective_channel(130, 52, {"radius": r, "x": 40.0, "y": 26.0, "motion": "imposed", "axis": 1,
                                         "amp": r / 2, "freq": 0.004, "phase": np.pi / 2, "u_ref": 0.048,
                                         "d_ref": 2 * r})


def _convective_lone_column():
    # nx = 2 * 64 + 1: the outlet column is a tile column of its own and the
    # ring of the tiles west of it; random populations so that the outlet
    # record differs row by row, a pitching ellipse near the outlet, no-slip
    # and moving walls
    p = wl.mixed_bc_box(129, 37, seed=15, west="velocity", east="convective", south="noslip", north="velocity",
                        tau=0.6, body={"shape": "ellipse", "radius": 7.0, "radius_b": 3.5, "x": 112.4,
                                       "y": 17.7, "theta": 0.3, "motion": "imposed", "axis": 2, "amp": 0.4,
                                       "freq": 0.02, "u_ref": 0.05, "d_ref": 7.0})
    p["bc"]["east"] = {"kind": "convective", "u": (0.31, 0.0)}
    p["f0"] = wl.random_populations(129, 37, seed=16, amp=0.02, u_amp=0.03)
    return p


def _convective_tiny_bgk():
    # smaller than one tile, BGK collision
    p = _convective_channel(7, 5, None, u=0.03, seed=17)
    p["collision"] = "bgk"
    p["f0"] = wl.random_populations(7, 5, seed=18, amp=0.02, u_amp=0.03)
    return p


CASES = {
    "tiny_walls": _tiny_walls,
    "periodic_x_symmetry_y": _periodic_x_symmetry_y,
    "channel_imposed": _channel_imposed,
    "fixed_ellipse": _fixed_ellipse,
    "pitching_rectangle_symmetry": _pitching_rectangle_symmetry,
    "periodic_no_body": lambda: _periodic_random(97, 70),
    "periodic_narrow_fixed_disk": lambda: _periodic_random(40, 30, {"radius": 5.3, "x": 36.2, "y": 27.9,
                                                                     "motion": "fixed"}),
    "periodic_tiny": lambda: _periodic_random(5, 4),
    "ragged_walls": _ragged_walls,
    "bgk_channel": _bgk_channel,
    "paper_channel_cosine": _paper_channel_cosine,
    "convective_lone_column": _convective_lone_column,
    "convective_tiny_bgk": _convective_tiny_bgk,
}


def _make(p, precision, kernel, hist=512):
    import paper_1905_05110_gb300 as vp
    sim = vp.Simulation(p, precision=precision, history_capacity=hist)
    if "f0" in p:
        sim.set_populations(p["f0"])
    else:
        sim.init_from_problem()
    if kernel == "fused2":
        sim.set_launch("fused2", 128, 1)
    else:
        sim.set_launch("scalar40", 256, 1)
    return sim


def _same_run(p, precision, steps_two=(5, 70, 21)):
    one = _make(p, precision, "scalar40")
    two = _make(p, precision, "fused2")
    n = sum(steps_two)
    one.step(n)
    for k in steps_two:   # single steps, graphs of two-step launches, single steps
        two.step(k)
    return one, two, n


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_two_step_kernel_equals_one_step_kernel_bitwise(case, precision):
    p = CASES[case]()
    one, two, n = _same_run(p, precision)
    assert np.array_equal(one.populations(), two.populations())
    assert two.launch()[0] == "fused2"
    if p.get("body"):
        h1, h2 = one.history(), two.history()
        assert np.array_equal(h1[:, REC["n_solid"]], h2[:, REC["n_solid"]])
        for key in ("t", "x", "y", "theta", "vx", "vy", "omega"):
            assert np.array_equal(h1[:, REC[key]], h2[:, REC[key]]), key
        for key in ("fx", "fy", "torque", "fpen_x", "fpen_y", "tpen"):
            assert rel_err(h2[:, REC[key]], h1[:, REC[key]]) < 1e-9, key
        q1, v1 = one.body_state()
        q2, v2 = two.body_state()
        assert np.array_equal(q1, q2) and np.array_equal(v1, v2)
    one.close()
    two.close()


@pytest.mark.parametrize("case", ["channel_imposed", "paper_channel_cosine"])
def test_two_step_kernel_matches_oracle(case):
    p = CASES[case]()
    gpu, orc = make_pair(p, "f32")
    gpu.set_launch("fused2", 128, 1)
    gpu.step(96)
    orc.step(96)
    assert dev_err(gpu.populations(), orc.populations()) < 1e-4
    hg, ho = gpu.history(), orc.history()
    assert np.array_equal(hg[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    for key in ("fx", "fy", "torque"):
        assert rel_err(hg[:, REC[key]], ho[:, REC[key]]) < 1e-3, key
    gpu.close()


@pytest.mark.parametrize("case", ["channel_imposed", "paper_channel_cosine"])
def test_two_step_kernel_launch_count_checkpoint_and_autotune(case, tmp_path):
    p = CASES[case]()
    sim = _make(p, "f32", "fused2")
    l0 = sim.launches
    sim.step(64)   # two graphs: a lookahead and 16 two-step launches each
    assert sim.launches - l0 == 34
    path = str(tmp_path / "two.ckpt")
    sim.save(path)
    sim.step(64)
    ref_f, ref_h = sim.populations(), sim.history(64, 64)
    sim.load(path)
    sim.step(64)
    assert np.array_equal(sim.populations(), ref_f)
    assert np.array_equal(sim.history(64, 64), ref_h)
    f_before = sim.populations()
    sim.autotune(8)
    assert np.array_equal(sim.populations(), f_before)
    sim.close()


def test_two_step_kernel_refusals():
    import paper_1905_05110_gb300 as vp
    cases = []
    cases.append((_channel_imposed(), "f64"))
    free = _channel_imposed()
    free["body"] = dict(free["body"], motion="free", mass=600.0, inertia=3e4, dof_mask=2)
    cases.append((free, "f32"))
    multi = _channel_imposed()
    multi["bodies"] = [multi["body"], dict(multi["body"], x=200.0, motion="fixed")]
    cases.append((multi, "f32"))
    for p, prec in cases:
        sim = vp.Simulation(p, precision=prec, history_capacity=64)
        with pytest.raises(vp.VplbmError) as ei:
            sim.set_launch("fused2", 128, 1)
        assert ei.value.status == 6
        sim.close()


def test_full_size_headline_two_step_kernel_equals_one_step_kernel():
    # The oscillating disk at its full 2048 x 1024 size, in the launch
    # configuration the benchmark times (two-step launches in 32-step graphs,
    # single steps on the 40-register kernel): bitwise the one-step kernel's
    # populations, whose full-size step is checked against the oracle node by
    # node in test_gpu_parity.
    p = wl.oscillating_disk()
    one = _make(p, "f32", "scalar40", hist=256)
    two = _make(p, "f32", "fused2", hist=256)
    one.step(70)
    for k in (3, 64, 3):
        two.step(k)
    assert np.array_equal(one.populations(), two.populations())
    h1, h2 = one.history(), two.history()
    assert np.array_equal(h1[:, REC["n_solid"]], h2[:, REC["n_solid"]])
    for key in ("fx", "fy", "torque"):
        assert rel_err(h2[:, REC[key]], h1[:, REC[key]]) < 1e-9, key
    one.close()
    two.close()


def test_full_size_paper_cylinder_two_step_kernel_equals_one_step_kernel():
    # The oscillating cylinder of Sec. 3.1 at its full 1230 x 410 size
    # (velocity inlet, convective outlet, symmetry walls, cosine law):
    # two-step launches in 32-step graphs between single steps, bitwise the
    # one-step kernel's populations and solid-node counts.
    p = wl.paper_oscillating_cylinder()
    one = _make(p, "f32", "scalar40", hist=256)
    two = _make(p, "f32", "fused2", hist=256)
    one.step(134)
    for k in (3, 64, 3, 64):
        two.step(k)
    assert np.array_equal(one.populations(), two.populations())
    h1, h2 = one.history(), two.history()
    assert np.array_equal(h1[:, REC["n_solid"]], h2[:, REC["n_solid"]])
    for key in ("fx", "fy", "torque"):
        assert rel_err(h2[:, REC[key]], h1[:, REC[key]]) < 1e-9, key
    one.close()
    two.close()


# (first step, steps in one call) -> launches the call must make, by kind:
# every call of 4 or more steps runs as pairs of two-step launches after one
# lookahead launch, but for its last nsteps mod 4 steps and, for more than
# 32 steps from an odd step, its first step (which takes it to an even step
# for a 32-step graph).
DISPATCH = {
    (1, 20): {"two_step": 10, "lookahead": 1, "one_step": 0},
    (0, 20): {"two_step": 10, "lookahead": 1, "one_step": 0},
    (1, 7): {"two_step": 2, "lookahead": 1, "one_step": 3},
    (3, 2): {"two_step": 0, "lookahead": 0, "one_step": 2},
    (1, 32): {"two_step": 16, "lookahead": 1, "one_step": 0},
    (1, 33): {"two_step": 16, "lookahead": 1, "one_step": 1},
    (3, 50): {"two_step": 24, "lookahead": 2, "one_step": 2},
}


@pytest.mark.parametrize("case", ["channel_imposed", "paper_channel_cosine", "periodic_x_symmetry_y"])
@pytest.mark.parametrize("precision", ["f32", "f16"])
@pytest.mark.parametrize("start,n", list(DISPATCH))
def test_step_call_runs_two_step_pairs_from_any_step(case, precision, start, n):
    # One call of n steps from step `start` against n calls of one step
    # (each a single launch of the one-step kernel): the same populations
    # bit for bit, the same poses and solid-node counts, and the launches
    # the dispatch rule gives.
    p = CASES[case]()
    one = _make(p, precision, "fused2")
    two = _make(p, precision, "fused2")
    one.step(start)
    two.step(start)
    for _ in range(n):
        one.step(1)
    k0 = two.kernel_launches()
    two.step(n)
    k1 = two.kernel_launches()
    made = {k: k1[k] - k0[k] for k in k1}
    assert made == dict(DISPATCH[(start, n)], tma=0)
    assert np.array_equal(one.populations(), two.populations())
    if p.get("body"):
        h1, h2 = one.history(), two.history()
        for key in ("t", "x", "y", "theta", "vx", "vy", "omega", "n_solid"):
            assert np.array_equal(h1[:, REC[key]], h2[:, REC[key]]), key
        for key in ("fx", "fy", "torque"):
            assert rel_err(h2[:, REC[key]], h1[:, REC[key]]) < 1e-9, key
        q1, v1 = one.body_state()
        q2, v2 = two.body_state()
        assert np.array_equal(q1, q2) and np.array_equal(v1, v2)
    one.close()
    two.close()


def test_launch_counts_by_kind_sum_to_launch_count():
    p = CASES["channel_imposed"]()
    sim = _make(p, "f32", "fused2")
    for n in (3, 20, 64, 5):
        sim.step(n)
    k = sim.kernel_launches()
    assert sum(k.values()) == sim.launches
    sim.set_launch("scalar40", 256, 1)
    k0, l0 = sim.kernel_launches(), sim.launches
    sim.step(40)
    k1 = sim.kernel_launches()
    assert k1["one_step"] - k0["one_step"] == 40 == sim.launches - l0
    sim.close()
