"""Several bodies in one lattice: the GPU path (through the C ABI) against
the FP64 oracle, body by body.

Eq. (2) is applied per body (a node is solid for the first listed body
whose chi holds there, with that body's rigid velocity); each body's force
and torque (Eqs. 25-27) sum its own solid nodes; each body has its own
record and motion.  Tolerances as in test_gpu_parity: populations as
deviations from rest, 1e-12 (FP64) / 1e-4 (FP32) / 5e-2 (FP16) over runs of
about a hundred steps; forces 1e-10 (FP64) / 1e-3 (FP32) of their scale;
the solid-node count of every body exactly.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from helpers import REC, dev_err, make_pair, rel_err

pytestmark = pytest.mark.gpu

RUN_TOL = {"f64": 1e-12, "f32": 1e-4, "f16": 5e-2}
FORCE_TOL = {"f64": 1e-10, "f32": 1e-3}
POSE_TOL = {"f64": 1e-12, "f32": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _library(gpu_library):
    return gpu_library


def _channel(nx, ny, bodies, tau=0.62):
    p = wl.mixed_bc_box(nx, ny, seed=4, west="velocity", east="zerograd", south="noslip", north="noslip",
                        tau=tau)
    p["s"] = wl.paper_rates(tau)
    p["bc"]["west"] = {"kind": "velocity", "u": (0.05, 0.0)}
    p["init"] = {"rho": 1.0, "u": (0.05, 0.0)}
    p["bodies"] = bodies
    return p


def _mixed(nx=160, ny=72):
    """A fixed disk, a pitching ellipse and a free rectangle, in a row."""
    a, b = 6.0, 3.5
    m = 4.0 * a * b * 1.2
    return _channel(nx, ny, [
        {"radius": 7.3, "x": 30.37, "y": 36.21, "motion": "fixed", "u_ref": 0.05, "d_ref": 14.6},
        {"shape": "ellipse", "radius": 10.0, "radius_b": 4.0, "x": 75.13, "y": 33.71, "theta": 0.3,
         "motion": "imposed", "axis": 2, "amp": 0.4, "freq": 0.01, "u_ref": 0.05, "d_ref": 8.0},
        {"shape": "rectangle", "radius": a, "radius_b": b, "x": 118.31, "y": 38.17, "theta": 0.2,
         "omega": 0.002, "motion": "free", "mass": m, "inertia": m * (a * a + b * b) / 3.0, "dof_mask": 7,
         "stiff": (0.0, 2e-3, 0.0), "q0": (0.0, 36.0, 0.0), "u_ref": 0.05, "d_ref": 2 * b},
    ])


def _overlap(nx=90, ny=64):
    """A disk and a rectangle that overlap (the disk, listed first, owns the
    shared nodes) and a free disk whose node range meets theirs."""
    r = 5.0
    return _channel(nx, ny, [
        {"radius": 8.0, "x": 40.3, "y": 31.7, "motion": "fixed", "u_ref": 0.05, "d_ref": 16.0},
        {"shape": "rectangle", "radius": 9.0, "radius_b": 3.0, "x": 48.1, "y": 33.2, "theta": 0.4,
         "motion": "imposed", "axis": 1, "amp": 1.0, "freq": 0.01},
        {"radius": r, "x": 66.4, "y": 30.1, "vy": 0.002, "motion": "free", "mass": 1.5 * np.pi * r * r,
         "inertia": 0.75 * np.pi * r ** 4, "dof_mask": 7, "u_ref": 0.05, "d_ref": 2 * r},
    ])


def _four(nx=128, ny=96):
    """Four free disks (the most a lattice holds) in a periodic box."""
    bodies = []
    for k, (x, y) in enumerate([(30.3, 25.7), (94.6, 28.2), (33.1, 70.4), (91.8, 69.9)]):
        r = 5.0 + 0.7 * k
        m = 1.5 * np.pi * r * r
        bodies.append({"radius": r, "x": x, "y": y, "vx": 0.003 * (k - 1.5), "vy": 0.002, "motion": "free",
                       "mass": m, "inertia": 0.5 * m * r * r, "dof_mask": 7, "u_ref": 0.05, "d_ref": 2 * r})
    p = wl.periodic_box(nx, ny, tau=0.7, g_fluid=(1e-5, 0.0))
    p["bodies"] = bodies
    return p


CONFIGS = {"mixed": _mixed, "overlap": _overlap, "four": _four}


def _pair(config, precision, hist_cap=4096):
    p = CONFIGS[config]()
    if config == "four":
        f0 = wl.random_populations(p["nx"], p["ny"], seed=17, amp=0.02, u_amp=0.03)
        return p, *make_pair(p, precision, hist_cap=hist_cap, f0=f0)
    return p, *make_pair(p, precision, hist_cap=hist_cap)


def _check_records(gpu, orc, nb, precision):
    for k in range(nb):
        hg, ho = gpu.history(body=k), orc.history(body=k)
        assert np.array_equal(hg[:, REC["n_solid"]], ho[:, REC["n_solid"]]), k
        assert np.all(ho[:, REC["n_solid"]] > 0), k
        for key in ("fx", "fy", "torque", "fpen_x", "fpen_y", "tpen"):
            assert rel_err(hg[:, REC[key]], ho[:, REC[key]]) < FORCE_TOL[precision], (k, key)
        for key in ("x", "y", "theta", "vx", "vy", "omega"):
            scale = max(1.0, np.max(np.abs(ho[:, REC[key]])))
            assert np.max(np.abs(hg[:, REC[key]] - ho[:, REC[key]])) <= POSE_TOL[precision] * scale, (k, key)
        q, v = gpu.body_state(k)
        qo, vo = orc.body_state(k)
        assert np.allclose(q, qo, rtol=0, atol=POSE_TOL[precision] * 100) and np.allclose(
            v, vo, rtol=0, atol=POSE_TOL[precision]), k


@pytest.mark.parametrize("config", list(CONFIGS))
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_several_bodies_match_oracle(config, precision):
    p, gpu, orc = _pair(config, precision)
    nb = len(p["bodies"])
    assert gpu.nbodies == nb
    steps = 120   # graphs of 32 steps and single launches
    gpu.step(steps)
    orc.step(steps)
    assert dev_err(gpu.populations(), orc.populations()) < RUN_TOL[precision]
    gr, gx, gy = gpu.fields()
    orr, ox, oy = orc.fields()
    assert rel_err(gx, ox) < RUN_TOL[precision] and rel_err(gy, oy) < RUN_TOL[precision]
    _check_records(gpu, orc, nb, precision)
    gpu.close()


def test_overlapping_bodies_first_listed_owns_the_shared_nodes():
    # The oracle's ownership map against a count on the host: the disk
    # (listed first) keeps every node inside it; the rectangle gets its own
    # nodes outside the disk only.  The GPU counts agree with it exactly.
    p, gpu, orc = _pair("overlap", "f32")
    chi = orc.chi()
    X, Y = np.meshgrid(np.arange(p["nx"], dtype=float), np.arange(p["ny"], dtype=float))
    d = p["bodies"][0]
    in_disk = (X - d["x"]) ** 2 + (Y - d["y"]) ** 2 <= d["radius"] ** 2
    assert np.all(chi[in_disk] == 1)
    r = p["bodies"][1]
    c, s = np.cos(r["theta"]), np.sin(r["theta"])
    u = (X - r["x"]) * c + (Y - r["y"]) * s
    v = (Y - r["y"]) * c - (X - r["x"]) * s
    in_rect = (np.abs(u) <= r["radius"]) & (np.abs(v) <= r["radius_b"])
    assert np.any(in_rect & in_disk)   # they do overlap
    assert np.array_equal(chi == 2, in_rect & ~in_disk)
    gpu.step(1)
    orc.step(1)
    for k in range(3):
        assert gpu.history(0, 1, body=k)[0, REC["n_solid"]] == orc.history(0, 1, body=k)[0, REC["n_solid"]]
    assert gpu.history(0, 1, body=1)[0, REC["n_solid"]] == np.sum(in_rect & ~in_disk)
    gpu.close()


@pytest.mark.parametrize("launch", [("scalar", 64, 4), ("scalar48", 32, 8), ("scalar40", 128, 2),
                                    ("scalar40", 32, 4)])
def test_several_bodies_every_register_budget_and_block_shape(launch):
    p, gpu, orc = _pair("mixed", "f32")
    gpu.set_launch(*launch)
    gpu.step(70)
    orc.step(70)
    assert dev_err(gpu.populations(), orc.populations()) < RUN_TOL["f32"]
    _check_records(gpu, orc, 3, "f32")
    gpu.close()


def test_several_bodies_fp16_storage():
    p, gpu, orc = _pair("mixed", "f16")
    gpu.step(60)
    orc.step(60)
    assert dev_err(gpu.populations(), orc.populations()) < RUN_TOL["f16"]
    for k in (0, 1):   # prescribed bodies: the same solid sets
        assert np.array_equal(gpu.history(body=k)[:, REC["n_solid"]], orc.history(body=k)[:, REC["n_solid"]])
    gpu.close()


def test_doubled_periodic_box_with_two_bodies_matches_one():
    # GPU counterpart of the oracle pin: two copies of a free body L apart in
    # a 2L-periodic box over an L-periodic state evolve like one body in the
    # L box (up to the rounding of the copy's lever arms).
    import paper_1905_05110_gb300 as vp
    L, ny = 64, 48
    body = {"radius": 6.3, "x": 27.4, "y": 23.2, "vy": 0.003, "omega": 0.002, "motion": "free",
            "mass": 400.0, "inertia": 8000.0, "stiff": (0.0, 2e-3, 0.0), "q0": (0.0, 24.0, 0.0),
            "dof_mask": 7, "u_ref": 0.04, "d_ref": 12.6}
    one = wl.periodic_box(L, ny, tau=0.7, body=body, g_fluid=(1e-5, 0.0))
    two = wl.periodic_box(2 * L, ny, tau=0.7, g_fluid=(1e-5, 0.0))
    two["bodies"] = [body, dict(body, x=body["x"] + L)]
    f0 = wl.random_populations(L, ny, seed=41, amp=0.02, u_amp=0.03)
    a = vp.Simulation(one, precision="f64", history_capacity=256)
    a.set_populations(f0)
    b = vp.Simulation(two, precision="f64", history_capacity=256)
    b.set_populations(np.concatenate([f0, f0], axis=2))
    a.step(100)
    b.step(100)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fb[:, :, :L] - fa)) < 1e-12
    assert np.max(np.abs(fb[:, :, L:] - fa)) < 1e-12
    ha = a.history()
    for k in (0, 1):
        hb = b.history(body=k).copy()
        hb[:, REC["x"]] -= k * L
        assert np.allclose(hb, ha, rtol=1e-9, atol=1e-13), k
    a.close()
    b.close()


def test_several_bodies_checkpoint_resume_and_autotune_are_exact(tmp_path):
    p, gpu, orc = _pair("mixed", "f32", hist_cap=256)
    gpu.step(40)
    path = str(tmp_path / "multi.ckpt")
    gpu.save(path)
    gpu.step(50)
    ref_f = gpu.populations()
    ref_h = [gpu.history(40, 50, body=k) for k in range(3)]
    gpu.load(path)
    gpu.step(50)
    assert np.array_equal(gpu.populations(), ref_f)
    for k in range(3):
        assert np.array_equal(gpu.history(40, 50, body=k), ref_h[k])
    # autotune leaves the state where it was
    f_before = gpu.populations()
    states = [gpu.body_state(k) for k in range(3)]
    gpu.autotune(8)
    assert gpu.launch()[0] != "tma"
    assert np.array_equal(gpu.populations(), f_before)
    for k in range(3):
        q, v = gpu.body_state(k)
        assert np.array_equal(q, states[k][0]) and np.array_equal(v, states[k][1])
    gpu.close()


def test_several_bodies_refusals_and_queries():
    import paper_1905_05110_gb300 as vp
    p = _mixed(160, 72)
    sim = vp.Simulation(p, precision="f32", history_capacity=64)
    assert vp.vplbm_get_num_bodies(sim.ctx) == 3
    with pytest.raises(vp.VplbmError) as ei:
        sim.set_launch("tma")
    assert ei.value.status == 6
    with pytest.raises(vp.VplbmError) as ei:
        sim.history(0, 0, body=3)
    assert ei.value.status == 1
    with pytest.raises(vp.VplbmError) as ei:
        sim.body_state(-1)
    assert ei.value.status == 1
    sim.close()
    sim = vp.Simulation(p, precision="f64", history_capacity=64)
    sim.init_from_problem()
    with pytest.raises(vp.VplbmError) as ei:
        sim.adjoint(10, 5)
    assert ei.value.status == 6
    sim.close()
    lat = vp.lattice_desc(p, "f32", [])
    five = [vp.body_desc(dict(p["bodies"][0], x=20.0 + 25 * k)) for k in range(5)]
    with pytest.raises(vp.VplbmError) as ei:
        vp.vplbm_create_bodies(lat, five, 64)
    assert ei.value.status == 1
    with pytest.raises(vp.VplbmError) as ei:
        vp.vplbm_create_bodies(lat, [], 64)
    assert ei.value.status == 1
    # a single-body context reports one body and body 0 only
    one = vp.Simulation(dict(p, bodies=None, body=p["bodies"][0]), precision="f32", history_capacity=64)
    assert vp.vplbm_get_num_bodies(one.ctx) == 1
    with pytest.raises(vp.VplbmError):
        one.history(0, 0, body=1)
    one.close()


def _mixed_bgk():
    p = _mixed()
    p["collision"] = "bgk"
    return p


def _mixed_paper_walls():
    # the paper's channel boundaries: symmetry walls and a convective outlet
    p = _mixed()
    p["bc"]["south"] = {"kind": "symmetry"}
    p["bc"]["north"] = {"kind": "symmetry"}
    p["bc"]["east"] = {"kind": "convective", "u": (0.05, 0.0)}
    return p


@pytest.mark.parametrize("variant", ["bgk", "paper_walls"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_several_bodies_with_bgk_and_with_the_papers_boundaries(variant, precision):
    p = _mixed_bgk() if variant == "bgk" else _mixed_paper_walls()
    gpu, orc = make_pair(p, precision)
    gpu.step(100)
    orc.step(100)
    assert dev_err(gpu.populations(), orc.populations()) < RUN_TOL[precision]
    _check_records(gpu, orc, 3, precision)
    gpu.close()
