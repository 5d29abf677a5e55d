"""The node-pair kernel (FP32 or FP16 storage, two x-adjacent nodes per
thread) against the one-node kernel and the FP64 oracle.

A pair runs the MRT update in the lane form on paired FP32 instructions,
each lane rounding as the one-node update does, and its body blocks are the
one-node kernel's; so populations, records and poses must equal those of
the one-node kernel at the same block shape bit for bit, over every boundary
kind, ragged sizes and moving bodies.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import REC, dev_err, make_pair, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library(gpu_library):
    return gpu_library


def _channel_imposed():
    return wl.oscillating_disk(nx=300, ny=130, diameter=20.0, x_c=61.3)


def _fixed_ellipse():
    p = wl.mixed_bc_box(162, 83, seed=7, west="velocity", east="zerograd", south="noslip", north="noslip", tau=0.6,
                        body={"shape": "ellipse", "radius": 14.0, "radius_b": 6.0, "x": 70.3, "y": 41.6,
                              "theta": 0.4, "motion": "fixed", "u_ref": 0.05, "d_ref": 12.0})
    p["init"] = {"rho": 1.0, "u": (0.03, 0.0)}
    return p


def _pitching_rectangle_symmetry():
    p = wl.mixed_bc_box(150, 70, seed=8, west="velocity", east="zerograd", south="symmetry", north="symmetry",
                        tau=0.62, body={"shape": "rectangle", "radius": 9.0, "radius_b": 4.0, "x": 60.2, "y": 35.3,
                                        "theta": 0.2, "motion": "imposed", "axis": 2, "amp": 0.5, "freq": 0.01,
                                        "u_ref": 0.05, "d_ref": 8.0})
    p["bc"]["west"] = {"kind": "velocity", "u": (0.05, 0.0)}
    p["init"] = {"rho": 1.0, "u": (0.05, 0.0)}
    return p


def _periodic_random(nx, ny, body=None):
    p = wl.periodic_box(nx, ny, tau=0.7, body=body, g_fluid=(1e-5, 2e-6))
    p["f0"] = wl.random_populations(nx, ny, seed=nx + ny, amp=0.02, u_amp=0.03)
    return p


def _ragged_walls():
    return wl.mixed_bc_box(130, 37, seed=11, west="velocity", east="velocity", south="velocity", north="noslip",
                           tau=0.66, body={"radius": 6.2, "x": 40.7, "y": 18.4, "motion": "imposed", "axis": 0,
                                           "amp": 2.0, "freq": 0.02, "u_ref": 0.03, "d_ref": 12.4},
                           rates=wl.random_rates(11))


def _convective_cosine():
    r = 6.0
    p = wl.mixed_bc_box(130, 52, seed=3, west="velocity", east="convective", south="symmetry", north="symmetry",
                        tau=0.56, body={"radius": r, "x": 40.0, "y": 26.0, "motion": "imposed", "axis": 1,
                                        "amp": r / 2, "freq": 0.004, "phase": np.pi / 2, "u_ref": 0.048,
                                        "d_ref": 2 * r})
    p["bc"]["west"] = {"kind": "velocity", "u": (0.048, 0.0)}
    p["bc"]["east"] = {"kind": "convective", "u": (0.048, 0.0)}
    p["init"] = {"rho": 1.0, "u": (0.048, 0.0)}
    return p


def _free_falling_disk():
    p = wl.sedimenting_disk(nx=128, ny=256, diameter=16)
    p["body"] = dict(p["body"], vx=0.003, vy=-0.002, omega=0.001)
    return p


def _tiny_walls():
    p = wl.mixed_bc_box(8, 5, seed=12, west="velocity", east="zerograd", south="noslip", north="velocity", tau=0.7)
    p["init"] = {"rho": 1.0, "u": (0.02, 0.0)}
    return p


CASES = {
    "channel_imposed": _channel_imposed,
    "fixed_ellipse": _fixed_ellipse,
    "pitching_rectangle_symmetry": _pitching_rectangle_symmetry,
    "periodic_no_body": lambda: _periodic_random(98, 70),
    "periodic_narrow_fixed_disk": lambda: _periodic_random(40, 30, {"radius": 5.3, "x": 36.2, "y": 27.9,
                                                                     "motion": "fixed"}),
    "ragged_walls": _ragged_walls,
    "convective_cosine": _convective_cosine,
    "free_falling_disk": _free_falling_disk,
    "tiny_walls": _tiny_walls,
}


def _make(p, kernel, bx, by, hist=512, precision="f16"):
    import paper_1905_05110_gb300 as vp
    sim = vp.Simulation(p, precision=precision, history_capacity=hist)
    if "f0" in p:
        sim.set_populations(p["f0"])
    else:
        sim.init_from_problem()
    sim.set_launch(kernel, bx, by)
    return sim


def _assert_same(one, two, p):
    assert np.array_equal(one.populations(), two.populations())
    if p.get("body"):
        h1, h2 = one.history(), two.history()
        assert np.array_equal(h1, h2)
        q1, v1 = one.body_state()
        q2, v2 = two.body_state()
        assert np.array_equal(q1, q2) and np.array_equal(v1, v2)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("shape", [(128, 2), (32, 8), (256, 1)])
@pytest.mark.parametrize("precision", ["f16", "f32"])
def test_pair_kernel_equals_one_node_kernel_bitwise(case, shape, precision):
    p = CASES[case]()
    one = _make(p, "scalar", *shape, precision=precision)
    two = _make(p, "pair", *shape, precision=precision)
    for n in (5, 70, 21):   # single launches and 32-step graphs
        one.step(n)
        two.step(n)
    _assert_same(one, two, p)
    assert two.launch()[0] == "pair"
    one.close()
    two.close()


@pytest.mark.parametrize("shape", [(64, 4), (64, 2), (32, 4), (128, 1)])
def test_pair_kernel_every_block_shape(shape):
    p = _channel_imposed()
    one = _make(p, "scalar40", *shape)
    two = _make(p, "pair", *shape)
    one.step(40)
    two.step(40)
    _assert_same(one, two, p)


@pytest.mark.parametrize("case", ["channel_imposed", "free_falling_disk", "convective_cosine"])
@pytest.mark.parametrize("precision,tol", [("f16", 5e-2), ("f32", 1e-4)])
def test_pair_kernel_matches_oracle(case, precision, tol):
    p = CASES[case]()
    gpu, orc = make_pair(p, precision)
    gpu.set_launch("pair", 128, 2)
    gpu.step(60)
    orc.step(60)
    assert dev_err(gpu.populations(), orc.populations()) < tol
    hg, ho = gpu.history(), orc.history()
    assert np.array_equal(hg[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    for key in ("fx", "fy"):
        assert rel_err(hg[:, REC[key]], ho[:, REC[key]]) < (5e-2 if precision == "f16" else 1e-3), key
    gpu.close()


@pytest.mark.parametrize("precision", ["f16", "f32"])
def test_full_size_headline_pair_kernel_equals_one_node_kernel(precision):
    # the oscillating disk at its full 2048 x 1024 size
    p = wl.oscillating_disk()
    one = _make(p, "scalar40", 256, 1, hist=128, precision=precision)
    two = _make(p, "pair", 256, 1, hist=128, precision=precision)
    for n in (3, 64):
        one.step(n)
        two.step(n)
    _assert_same(one, two, p)
    one.close()
    two.close()


def test_pair_kernel_refusals():
    import paper_1905_05110_gb300 as vp
    base = _channel_imposed()
    cases = [(base, "f64"), (dict(base, nx=301), "f16"), (dict(base, nx=301), "f32"), (dict(base, collision="bgk"), "f16")]
    multi = _channel_imposed()
    multi["bodies"] = [multi["body"], dict(multi["body"], x=200.0, motion="fixed")]
    cases.append((multi, "f16"))
    for p, prec in cases:
        sim = vp.Simulation(p, precision=prec, history_capacity=64)
        with pytest.raises(vp.VplbmError) as ei:
            sim.set_launch("pair", 128, 2)
        assert ei.value.status == 6, (prec, p["nx"])
        sim.close()


def test_pair_kernel_checkpoint_and_autotune(tmp_path):
    p = _channel_imposed()
    sim = _make(p, "pair", 128, 2)
    sim.step(40)
    path = str(tmp_path / "pair.ckpt")
    sim.save(path)
    sim.step(40)
    ref_f, ref_h = sim.populations(), sim.history(40, 40)
    sim.load(path)
    sim.step(40)
    assert np.array_equal(sim.populations(), ref_f)
    assert np.array_equal(sim.history(40, 40), ref_h)
    f_before = sim.populations()
    sim.autotune(8)
    assert np.array_equal(sim.populations(), f_before)
    sim.close()
