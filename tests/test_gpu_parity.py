"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (max |gpu - oracle| / max |oracle| per field; populations are
compared as deviations from rest, f - w rho0):
  - FP64 storage and arithmetic: 1e-12 on populations and fields, forces to
    1e-10 of their scale (sums of a few hundred terms in another order).
  - FP32 deviation storage: one step from a common state 2e-6 (a handful of
    FP32 roundings of an O(u) deviation); runs of hundreds of steps 1e-4.
  - FP16 deviation storage: one step 2e-3 (11-bit mantissa of the stored
    deviation); runs 5e-2.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from helpers import REC, dev_err, make_pair, moving_bodies, rel_err

pytestmark = pytest.mark.gpu

BC_SETS = [
    ("periodic", "periodic", "periodic", "periodic"),
    ("velocity", "zerograd", "noslip", "velocity"),
    ("noslip", "noslip", "periodic", "periodic"),
    ("velocity", "velocity", "noslip", "noslip"),
    ("zerograd", "zerograd", "velocity", "noslip"),
    ("periodic", "periodic", "velocity", "velocity"),
    ("velocity", "zerograd", "symmetry", "symmetry"),
    ("periodic", "periodic", "symmetry", "noslip"),
    ("velocity", "convective", "noslip", "symmetry"),
    ("noslip", "convective", "velocity", "velocity"),
]

ONE_STEP_TOL = {"f64": 1e-13, "f32": 2e-6, "f16": 2e-3}
RUN_TOL = {"f64": 1e-12, "f32": 1e-4, "f16": 5e-2}


@pytest.fixture(scope="module", autouse=True)
def _library(gpu_library):
    return gpu_library


def _box(nx, ny, bcs, seed, body=None, tau=0.7):
    w, e, s, n = bcs
    p = wl.mixed_bc_box(nx, ny, seed=seed, west=w, east=e, south=s, north=n, tau=tau, body=body,
                        rates=wl.random_rates(seed))
    if e == "convective":
        p["bc"]["east"] = {"kind": "convective", "u": (0.31, 0.0)}
    return p


@pytest.mark.parametrize("bcs", BC_SETS)
@pytest.mark.parametrize("size", [(67, 45), (5, 4), (130, 3)])
@pytest.mark.parametrize("precision", ["f64", "f32", "f16"])
def test_steps_from_random_state_every_boundary(bcs, size, precision):
    nx, ny = size
    p = _box(nx, ny, bcs, seed=nx + ny)
    f0 = wl.random_populations(nx, ny, seed=11, amp=0.03, u_amp=0.05)
    if precision != "f64":   # both sides start from the stored (rounded) state
        gpu, _ = make_pair(p, precision, init=None, f0=f0)
        f0 = gpu.populations()
    gpu, orc = make_pair(p, precision, f0=f0)
    for n in (1, 2):
        gpu.step(1)
        orc.step(1)
        tol = ONE_STEP_TOL[precision] * (3 if n == 2 else 1)
        assert dev_err(gpu.populations(), orc.populations()) < tol
        gr, gx, gy = gpu.fields()
        orr, ox, oy = orc.fields()
        assert rel_err(gr - 1, orr - 1) < 10 * tol
        assert rel_err(gx, ox) < 10 * tol and rel_err(gy, oy) < 10 * tol


@pytest.mark.parametrize("motion", ["fixed", "imposed", "free"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_body_runs_match_oracle(motion, precision):
    nx, ny = 97, 70
    body = moving_bodies(nx, ny)[motion]
    p = _box(nx, ny, ("velocity", "zerograd", "noslip", "noslip"), seed=5, body=body, tau=0.62)
    p["bc"]["west"] = {"kind": "velocity", "u": (0.05, 0.0)}
    gpu, orc = make_pair(p, precision)
    steps = 150
    gpu.step(steps)
    orc.step(steps)
    tol = RUN_TOL[precision]
    assert dev_err(gpu.populations(), orc.populations()) < tol
    gr, gx, gy = gpu.fields()
    orr, ox, oy = orc.fields()
    assert rel_err(gx, ox) < tol and rel_err(gy, oy) < tol
    hg, ho = gpu.history(), orc.history()
    assert np.array_equal(hg[:, REC["t"]], np.arange(steps))
    assert np.array_equal(hg[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    ftol = 1e-10 if precision == "f64" else 1e-3
    for key in ("fx", "fy", "torque", "fpen_x", "fpen_y", "tpen"):
        assert rel_err(hg[:, REC[key]], ho[:, REC[key]]) < ftol, key
    ptol = 1e-12 if precision == "f64" else 1e-6
    for key in ("x", "y", "theta", "vx", "vy", "omega"):
        assert np.max(np.abs(hg[:, REC[key]] - ho[:, REC[key]])) <= ptol * max(1.0, np.max(np.abs(ho[:, REC[key]]))), key


def test_channel_fixed_disk_fp64_full_run():
    # 256 x 128 parabolic channel past a fixed disk, 2000 steps, FP64.
    p = wl.channel_fixed_disk()
    gpu, orc = make_pair(p, "f64")
    gpu.step(p["steps"])
    orc.step(p["steps"])
    gr, gx, gy = gpu.fields()
    orr, ox, oy = orc.fields()
    errs = {"f": rel_err(gpu.populations(), orc.populations()), "rho": rel_err(gr, orr),
            "ux": rel_err(gx, ox), "uy": rel_err(gy, oy), "rho-1": rel_err(gr - 1, orr - 1)}
    print("fp64 channel 2000 steps:", errs)
    # fields and populations 1e-12 of their scale; the density deviation
    # (10^3 smaller than rho) 1e-10 of its own scale
    assert errs["f"] < 1e-12 and errs["rho"] < 1e-12
    assert errs["ux"] < 1e-12 and errs["uy"] < 1e-12
    assert errs["rho-1"] < 1e-10
    hg, ho = gpu.history(), orc.history()
    assert np.max(np.abs(hg[:, REC["cd"]] - ho[:, REC["cd"]])) < 1e-10
    assert np.max(np.abs(hg[:, REC["cl"]] - ho[:, REC["cl"]])) < 1e-10


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_channel_fixed_disk_reduced_precision(precision):
    p = wl.channel_fixed_disk(steps=600)
    gpu, orc = make_pair(p, precision)
    gpu.step(p["steps"])
    orc.step(p["steps"])
    gr, gx, gy = gpu.fields()
    orr, ox, oy = orc.fields()
    tol = RUN_TOL[precision]
    assert rel_err(gx, ox) < tol and rel_err(gy, oy) < tol
    hg, ho = gpu.history(), orc.history()
    assert np.max(np.abs(hg[-100:, REC["cd"]] - ho[-100:, REC["cd"]])) < 50 * tol


FULL = {
    "oscillating_2048x1024": lambda: wl.oscillating_disk(),
    "sedimenting_1024x4096": lambda: wl.sedimenting_disk(),
    "adjoint_1024x512": lambda: wl.adjoint_disk(),
}


@pytest.mark.parametrize("name", sorted(FULL))
def test_full_size_one_step_every_launch_shape(name):
    # Full workload size: after a few GPU steps, one more step from the same
    # state on the GPU (each launch shape) and in the oracle, all nodes.
    import paper_1905_05110_gb300 as vp
    p = FULL[name]()
    gpu = vp.Simulation(p, precision="f32", history_capacity=64)
    gpu.init_from_problem()
    gpu.step(6)
    f0 = gpu.populations()
    q0, v0 = gpu.body_state()
    body = dict(p["body"])
    body.update(x=q0[0], y=q0[1], theta=q0[2], vx=v0[0], vy=v0[1], omega=v0[2])
    if body["motion"] == "imposed":
        body["motion"] = "fixed"   # one step: compare the state update, pose from history
    p1 = dict(p, body=body)
    orc = oracle.OracleSim(p1, hist_cap=4)
    orc.set_populations(f0)
    orc.step(1)
    ref = orc.populations()
    ref_h = orc.history(0, 1)[0]
    for kern, bx, by in vp_shapes():
        g = vp.Simulation(p1, precision="f32", history_capacity=4)
        g.set_launch(kern, bx, by)
        g.set_populations(f0)
        g.step(1)
        assert dev_err(g.populations(), ref) < ONE_STEP_TOL["f32"], (kern, bx, by)
        h = g.history(0, 1)[0]
        assert h[REC["n_solid"]] == ref_h[REC["n_solid"]]
        assert rel_err(h[[REC["fx"], REC["fy"]]], ref_h[[REC["fx"], REC["fy"]]]) < 1e-3
        g.close()
    del orc


SCALAR_SHAPES = [(128, 2), (256, 1), (64, 4), (32, 8), (128, 1), (64, 2), (32, 4)]


def vp_shapes():
    """Every kernel and block shape the runtime can launch."""
    return ([("tma", 0, 0)] + [("scalar48", bx, by) for bx, by in SCALAR_SHAPES]
            + [("scalar", bx, by) for bx, by in SCALAR_SHAPES]
            + [("scalar40", bx, by) for bx, by in SCALAR_SHAPES])


def test_fp64_full_size_two_steps():
    p = wl.oscillating_disk()
    gpu, orc = make_pair(p, "f64", hist_cap=8)
    gpu.step(2)
    orc.step(2)
    assert dev_err(gpu.populations(), orc.populations()) < 1e-13
    hg, ho = gpu.history(), orc.history()
    assert rel_err(hg[:, REC["fy"]], ho[:, REC["fy"]]) < 1e-10
    assert np.max(np.abs(hg[:, REC["y"]] - ho[:, REC["y"]])) < 1e-12


def test_deterministic_and_graph_equals_direct_launches():
    p = wl.oscillating_disk(nx=300, ny=160, diameter=24, x_c=80)
    import paper_1905_05110_gb300 as vp
    runs = []
    for mode in ("graph", "graph", "direct"):
        g = vp.Simulation(p, precision="f32", history_capacity=256)
        g.init_from_problem()
        if mode == "graph":
            g.step(96)
        else:
            for _ in range(96):
                g.step(1)
        runs.append((g.populations(), g.history()))
        g.close()
    for f, h in runs[1:]:
        assert np.array_equal(f, runs[0][0])
        assert np.array_equal(h, runs[0][1])


def test_launch_shapes_give_identical_fields_for_fixed_body():
    import paper_1905_05110_gb300 as vp
    p = wl.channel_fixed_disk(nx=200, ny=90, center=(50.3, 44.6), diameter=18)
    ref = None
    for bx, by in SCALAR_SHAPES:
        g = vp.Simulation(p, precision="f32", history_capacity=64)
        g.set_launch("scalar", bx, by)
        g.init_from_problem()
        g.step(40)
        f = g.populations()
        if ref is None:
            ref = f
        assert np.array_equal(f, ref), (bx, by)
        g.close()


def test_checkpoint_resume_is_bitwise(tmp_path):
    import paper_1905_05110_gb300 as vp
    p = wl.sedimenting_disk(nx=128, ny=256, diameter=16)
    a = vp.Simulation(p, precision="f32", history_capacity=128)
    a.init_from_problem()
    a.step(41)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(40)
    b = vp.Simulation(p, precision="f32", history_capacity=128)
    b.load(path)
    assert b.nstep == 41
    b.step(40)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.history(), b.history())


def test_history_ring_and_ranges():
    import paper_1905_05110_gb300 as vp
    p = wl.channel_fixed_disk(nx=64, ny=40, center=(20, 20), diameter=8)
    big = vp.Simulation(p, precision="f32", history_capacity=64)
    small = vp.Simulation(p, precision="f32", history_capacity=10)
    for g in (big, small):
        g.init_from_problem()
        g.step(25)
    with pytest.raises(vp.VplbmError) as ei:
        small.history(0, 5)
    assert ei.value.status == 7
    with pytest.raises(vp.VplbmError):
        big.history(20, 10)
    assert np.array_equal(small.history(15, 10), big.history(15, 10))


def test_nonfinite_state_is_reported_not_trapped():
    import paper_1905_05110_gb300 as vp
    p = wl.channel_fixed_disk(nx=64, ny=40, center=(20, 20), diameter=8)
    g = vp.Simulation(p, precision="f32", history_capacity=16)
    f = wl.random_populations(64, 40, seed=2)
    f[3, 10, 30] = np.nan
    g.set_populations(f)
    g.step(2)
    with pytest.raises(vp.VplbmError) as ei:
        g.sync()
    assert ei.value.status == 4
    # the context stays usable
    g.init_from_problem()
    g.step(3)
    g.sync()


def test_fields_dev_matches_host_fields():
    import torch
    import paper_1905_05110_gb300 as vp
    p = wl.oscillating_disk(nx=160, ny=96, diameter=16, x_c=40)
    g = vp.Simulation(p, precision="f32", history_capacity=16)
    g.init_from_problem()
    g.step(7)
    rho, ux, uy = g.fields()
    out = torch.empty((3, 96, 160), dtype=torch.float64, device="cuda")
    vp.vplbm_get_fields_dev(g.ctx, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
    g.sync()
    o = out.cpu().numpy()
    assert np.array_equal(o[0], rho) and np.array_equal(o[1], ux) and np.array_equal(o[2], uy)


def test_autotune_restores_state():
    import paper_1905_05110_gb300 as vp
    p = wl.oscillating_disk(nx=512, ny=256, diameter=20, x_c=100)
    g = vp.Simulation(p, precision="f32", history_capacity=64)
    g.init_from_problem()
    g.step(10)
    f = g.populations()
    h = g.history()
    shape = g.autotune(4)
    assert shape[0] == "tma" or shape in [tuple(s) for s in vp_shapes()]
    assert g.nstep == 10
    assert np.array_equal(g.populations(), f)
    assert np.array_equal(g.history(), h)


@pytest.mark.parametrize("bcs", BC_SETS)
@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_tma_kernel_steps_from_random_state(bcs, precision):
    # lattice the TMA-staged kernel accepts (nx a multiple of 8), ragged in
    # both directions against its 128 x 4 chunks, every boundary set
    import paper_1905_05110_gb300 as vp
    nx, ny = 264, 37
    body = moving_bodies(nx, ny)["free"]
    p = _box(nx, ny, bcs, seed=nx + ny, body=body)
    f0 = wl.random_populations(nx, ny, seed=12, amp=0.03, u_amp=0.05)
    g, _ = make_pair(p, precision, init=None, f0=f0)
    f0 = g.populations()
    gpu, orc = make_pair(p, precision, f0=f0)
    gpu.set_launch("tma")
    for n in (1, 2):
        gpu.step(1)
        orc.step(1)
        tol = ONE_STEP_TOL[precision] * (3 if n == 2 else 1)
        assert dev_err(gpu.populations(), orc.populations()) < tol
    hg, ho = gpu.history(), orc.history()
    assert np.array_equal(hg[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    assert rel_err(hg[:, REC["fx"]], ho[:, REC["fx"]]) < 1e-3


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_tma_kernel_matches_plain_kernel_over_a_run(precision):
    import paper_1905_05110_gb300 as vp
    p = wl.oscillating_disk(nx=392, ny=203, diameter=30, x_c=100)
    runs = {}
    for shape in (("tma", 0, 0), ("scalar", 128, 2)):
        g = vp.Simulation(p, precision=precision, history_capacity=256)
        g.set_launch(*shape)
        g.init_from_problem()
        g.step(150)
        runs[shape[0]] = (g.populations(), g.history())
        g.close()
    (fa, ha), (fb, hb) = runs["tma"], runs["scalar"]
    assert dev_err(fa, fb) < (1e-5 if precision == "f32" else 1e-2)
    assert np.array_equal(ha[:, REC["n_solid"]], hb[:, REC["n_solid"]])
    assert rel_err(ha[:, REC["cl"]], hb[:, REC["cl"]]) < (1e-3 if precision == "f32" else 5e-2)


def test_tma_bounded_wait_reports_timeout_and_context_survives():
    import paper_1905_05110_gb300 as vp
    p = wl.oscillating_disk(nx=256, ny=64, diameter=12, x_c=60)
    g = vp.Simulation(p, precision="f32", history_capacity=64)
    g.init_from_problem()
    g.set_launch("tma")
    vp.vplbm_inject_wait_timeout(g.ctx, True)
    g.step(1)
    with pytest.raises(vp.VplbmError) as ei:
        g.sync()
    assert ei.value.status == 5
    vp.vplbm_inject_wait_timeout(g.ctx, False)
    g.init_from_problem()
    g.step(40)
    g.sync()
    ref = vp.Simulation(p, precision="f32", history_capacity=64)
    ref.set_launch("tma")
    ref.init_from_problem()
    ref.step(40)
    assert np.array_equal(g.populations(), ref.populations())


# ---- single-relaxation-time (BGK) operator of Sec. 2.1 ------------------

@pytest.mark.parametrize("bcs", BC_SETS)
@pytest.mark.parametrize("size", [(67, 45), (130, 3)])
@pytest.mark.parametrize("precision", ["f64", "f32", "f16"])
def test_bgk_steps_from_random_state(bcs, size, precision):
    nx, ny = size
    p = _box(nx, ny, bcs, seed=nx + 2 * ny)
    p["collision"] = "bgk"
    f0 = wl.random_populations(nx, ny, seed=13, amp=0.03, u_amp=0.05)
    if precision != "f64":
        gpu, _ = make_pair(p, precision, init=None, f0=f0)
        f0 = gpu.populations()
    gpu, orc = make_pair(p, precision, f0=f0)
    for n in (1, 2):
        gpu.step(1)
        orc.step(1)
        tol = ONE_STEP_TOL[precision] * (3 if n == 2 else 1)
        assert dev_err(gpu.populations(), orc.populations()) < tol
        gr, gx, gy = gpu.fields()
        orr, ox, oy = orc.fields()
        assert rel_err(gr - 1, orr - 1) < 10 * tol
        assert rel_err(gx, ox) < 10 * tol and rel_err(gy, oy) < 10 * tol


@pytest.mark.parametrize("motion", ["imposed", "free"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_bgk_body_runs_match_oracle(motion, precision):
    nx, ny = 97, 70
    body = moving_bodies(nx, ny)[motion]
    p = _box(nx, ny, ("velocity", "zerograd", "noslip", "noslip"), seed=7, body=body, tau=0.62)
    p["collision"] = "bgk"
    p["s"] = [1.0 / 0.62] * 9
    p["bc"]["west"] = {"kind": "velocity", "u": (0.05, 0.0)}
    gpu, orc = make_pair(p, precision)
    steps = 150
    gpu.step(steps)
    orc.step(steps)
    tol = RUN_TOL[precision]
    assert dev_err(gpu.populations(), orc.populations()) < tol
    hg, ho = gpu.history(), orc.history()
    assert np.array_equal(hg[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    ftol = 1e-10 if precision == "f64" else 1e-3
    for key in ("fx", "fy", "torque", "fpen_x", "fpen_y", "tpen"):
        assert rel_err(hg[:, REC[key]], ho[:, REC[key]]) < ftol, key


def test_bgk_register_budgets_agree_and_unsupported_paths_refuse():
    import paper_1905_05110_gb300 as vp
    nx, ny = 300, 96
    body = moving_bodies(nx, ny)["imposed"]
    p = _box(nx, ny, ("velocity", "zerograd", "noslip", "noslip"), seed=9, body=body)
    p["collision"] = "bgk"
    p["bc"]["west"] = {"kind": "velocity", "u": (0.04, 0.0)}
    out = []
    for kern, bx, by in (("scalar", 256, 1), ("scalar48", 128, 2), ("scalar40", 64, 4)):
        sim = vp.Simulation(p, precision="f32", history_capacity=128)
        sim.set_launch(kern, bx, by)
        sim.init_from_problem()
        sim.step(40)
        out.append((sim.populations(), sim.history()))
        if kern == "scalar":
            with pytest.raises(vp.VplbmError) as ei:
                sim.set_launch("tma")
            assert ei.value.status == 6
            with pytest.raises(vp.VplbmError) as ei:
                sim.adjoint(10, 5)
            assert ei.value.status == 6
        sim.close()
    for pops, hist in out[1:]:
        assert np.array_equal(pops, out[0][0])
        assert np.array_equal(hist[:, REC["n_solid"]], out[0][1][:, REC["n_solid"]])
        assert rel_err(hist[:, REC["fy"]], out[0][1][:, REC["fy"]]) < 1e-5


# ---- symmetry walls (the oscillating-cylinder setup of Sec. 3.1) ----------

@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_symmetry_channel_with_oscillating_disk_matches_oracle(precision):
    nx, ny = 120, 50
    body = moving_bodies(nx, ny)["imposed"]
    p = wl.mixed_bc_box(nx, ny, seed=12, west="velocity", east="zerograd", south="symmetry",
                        north="symmetry", tau=0.56, body=body)   # the paper's rates for tau = 0.56
    p["bc"]["west"] = {"kind": "velocity", "u": (0.048, 0.0)}
    p["init"] = {"rho": 1.0, "u": (0.048, 0.0)}
    gpu, orc = make_pair(p, precision)
    gpu.step(120)
    orc.step(120)
    tol = RUN_TOL[precision]
    assert dev_err(gpu.populations(), orc.populations()) < tol
    hg, ho = gpu.history(), orc.history()
    assert np.array_equal(hg[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    ftol = 1e-10 if precision == "f64" else 1e-3
    for key in ("fx", "fy", "torque"):
        assert rel_err(hg[:, REC[key]], ho[:, REC[key]]) < ftol, key


def test_symmetry_rejected_where_not_defined():
    import paper_1905_05110_gb300 as vp
    p = _box(40, 20, ("velocity", "zerograd", "symmetry", "symmetry"), seed=1)
    p["bc"]["east"] = {"kind": "symmetry"}
    with pytest.raises(vp.VplbmError) as ei:
        vp.Simulation(p, precision="f32")
    assert ei.value.status == 6
    p = _box(40, 20, ("velocity", "zerograd", "symmetry", "symmetry"), seed=1,
             body=moving_bodies(40, 20)["imposed"])
    sim = vp.Simulation(p, precision="f64", history_capacity=64)
    sim.init_from_problem()
    with pytest.raises(vp.VplbmError) as ei:
        sim.adjoint(10, 5)
    assert ei.value.status == 6
    sim.close()


# ---- convective outlet (the oscillating-cylinder setup of Sec. 3.1) -------

def _paper_channel(nx, ny, body):
    """Velocity inlet, convective outlet, symmetry walls, as in Sec. 3.1."""
    p = wl.mixed_bc_box(nx, ny, seed=3, west="velocity", east="convective", south="symmetry",
                        north="symmetry", tau=0.56, body=body)
    p["bc"]["west"] = {"kind": "velocity", "u": (0.048, 0.0)}
    p["bc"]["east"] = {"kind": "convective", "u": (0.048, 0.0)}
    p["init"] = {"rho": 1.0, "u": (0.048, 0.0)}
    return p


@pytest.mark.parametrize("precision", ["f64", "f32", "f16"])
def test_paper_channel_with_cosine_oscillation_matches_oracle(precision):
    nx, ny = 130, 52
    r = 6.0
    body = {"radius": r, "x": 40.0, "y": 26.0, "motion": "imposed", "axis": 1, "amp": r / 2,
            "freq": 0.004, "phase": np.pi / 2, "u_ref": 0.048, "d_ref": 2 * r}
    p = _paper_channel(nx, ny, body)
    gpu, orc = make_pair(p, precision)
    gpu.step(150)
    orc.step(150)
    tol = RUN_TOL[precision]
    assert dev_err(gpu.populations(), orc.populations()) < tol
    gr, gx, gy = gpu.fields()
    orr, ox, oy = orc.fields()
    assert rel_err(gx, ox) < tol and rel_err(gy, oy) < tol
    hg, ho = gpu.history(), orc.history()
    assert np.array_equal(hg[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    if precision != "f16":
        ftol = 1e-10 if precision == "f64" else 1e-3
        for key in ("fx", "fy", "torque"):
            assert rel_err(hg[:, REC[key]], ho[:, REC[key]]) < ftol, key


def test_convective_outlet_state_survives_checkpoint_and_autotune(tmp_path):
    import paper_1905_05110_gb300 as vp
    p = _paper_channel(300, 40, None)
    a = vp.Simulation(p, precision="f32", history_capacity=128)
    a.init_from_problem()
    a.step(17)
    a.autotune(4)           # trial steps are undone, outlet state included
    assert a.nstep == 17
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(30)
    b = vp.Simulation(p, precision="f32", history_capacity=128)
    b.load(path)
    b.set_launch(*a.launch())
    b.step(30)
    assert np.array_equal(a.populations(), b.populations())
    c = vp.Simulation(p, precision="f32", history_capacity=128)
    c.set_launch(*a.launch())
    c.init_from_problem()
    c.step(47)
    assert np.array_equal(a.populations(), c.populations())


def test_convective_outlet_rejected_where_not_defined():
    import paper_1905_05110_gb300 as vp
    p = _paper_channel(60, 20, moving_bodies(60, 20)["imposed"])
    p["bc"]["west"] = {"kind": "convective", "u": (0.1, 0.0)}
    with pytest.raises(vp.VplbmError) as ei:
        vp.Simulation(p, precision="f32")
    assert ei.value.status == 6
    p = _paper_channel(60, 20, moving_bodies(60, 20)["imposed"])
    p["bc"]["east"] = {"kind": "convective", "u": (-0.1, 0.0)}
    with pytest.raises(vp.VplbmError) as ei:
        vp.Simulation(p, precision="f32")
    assert ei.value.status == 1
    p = _paper_channel(60, 20, moving_bodies(60, 20)["imposed"])
    sim = vp.Simulation(p, precision="f64", history_capacity=64)
    sim.init_from_problem()
    with pytest.raises(vp.VplbmError) as ei:
        sim.adjoint(10, 5)
    assert ei.value.status == 6
    sim.close()


# ---- elliptic body ---------------------------------------------------------

def _ellipse_body(motion, nx, ny, shape="ellipse"):
    a, b = 0.2 * ny, 0.09 * ny
    m = 2.0 * np.pi * a * b
    common = {"shape": shape, "radius": a, "radius_b": b, "u_ref": 0.05, "d_ref": 2 * b}
    if motion == "fixed":
        return dict(common, x=0.41 * nx + 0.13, y=0.52 * ny + 0.37, theta=0.5, motion="fixed")
    if motion == "imposed":   # pitching about its centre
        return dict(common, x=0.43 * nx + 0.21, y=0.47 * ny + 0.09, theta=0.3, motion="imposed", axis=2,
                    amp=0.4, freq=0.01, phase=0.0)
    return dict(common, x=0.45 * nx + 0.31, y=0.5 * ny + 0.17, theta=0.1, omega=0.004, vy=-0.002,
                motion="free", mass=m, inertia=m * (a * a + b * b) / 4, dof_mask=7,
                stiff=(0.0, 1e-3, 0.0), q0=(0.0, 0.5 * ny, 0.0))


@pytest.mark.parametrize("shape", ["ellipse", "rectangle"])
@pytest.mark.parametrize("motion", ["fixed", "imposed", "free"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_shaped_body_runs_match_oracle(shape, motion, precision):
    nx, ny = 97, 70
    p = _box(nx, ny, ("velocity", "zerograd", "noslip", "noslip"), seed=6,
             body=_ellipse_body(motion, nx, ny, shape), tau=0.62)
    p["s"] = wl.paper_rates(0.62)
    p["bc"]["west"] = {"kind": "velocity", "u": (0.05, 0.0)}
    gpu, orc = make_pair(p, precision)
    steps = 150
    gpu.step(steps)
    orc.step(steps)
    tol = RUN_TOL[precision]
    assert dev_err(gpu.populations(), orc.populations()) < tol
    hg, ho = gpu.history(), orc.history()
    assert np.array_equal(hg[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    ftol = 1e-10 if precision == "f64" else 1e-3
    for key in ("fx", "fy", "torque", "fpen_x", "fpen_y", "tpen"):
        assert rel_err(hg[:, REC[key]], ho[:, REC[key]]) < ftol, key
    ptol = 1e-12 if precision == "f64" else 1e-6
    for key in ("x", "y", "theta", "vx", "vy", "omega"):
        assert np.max(np.abs(hg[:, REC[key]] - ho[:, REC[key]])) <= ptol * max(1.0, np.max(np.abs(ho[:, REC[key]]))), key
    if motion != "fixed":
        assert np.ptp(hg[:, REC["n_solid"]]) > 0   # the solid set changes as it turns


def test_ellipse_with_equal_axes_is_the_disk_and_refusals():
    import paper_1905_05110_gb300 as vp
    nx, ny = 130, 66
    disk = {"radius": 9.3, "x": 52.37, "y": 31.61, "motion": "imposed", "axis": 1, "amp": 2.0, "freq": 0.01,
            "u_ref": 0.05, "d_ref": 18.6}
    ell = dict(disk, shape="ellipse", radius_b=9.3, theta=0.0)
    out = []
    for body in (disk, ell):
        p = _box(nx, ny, ("velocity", "zerograd", "noslip", "noslip"), seed=2, body=body)
        p["s"] = wl.paper_rates(0.7)
        sim = vp.Simulation(p, precision="f32", history_capacity=64)
        sim.init_from_problem()
        sim.step(40)
        out.append((sim.populations(), sim.history()))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1][:, REC["n_solid"]], out[1][1][:, REC["n_solid"]])
    p = _box(nx, ny, ("velocity", "zerograd", "noslip", "noslip"), seed=2, body=dict(ell, radius_b=0.0))
    with pytest.raises(vp.VplbmError) as ei:
        vp.Simulation(p, precision="f32")
    assert ei.value.status == 1
    p = _box(nx, ny, ("velocity", "zerograd", "noslip", "noslip"), seed=2, body=dict(ell, radius_b=4.0))
    sim = vp.Simulation(p, precision="f64", history_capacity=64)
    sim.init_from_problem()
    with pytest.raises(vp.VplbmError) as ei:
        sim.adjoint(10, 5)
    assert ei.value.status == 6
    sim.close()


def test_tall_lattice_takes_taller_blocks_within_the_grid_row_limit():
    # 40 x 65535: 256 x 1 blocks would need 65536 grid rows (65535 tile rows
    # and one body-block row); the context takes 128 x 2 and refuses 256 x 1.
    import paper_1905_05110_gb300 as vp
    p = wl.periodic_box(40, 65535, tau=0.7)
    sim = vp.Simulation(p, precision="f16", history_capacity=8)
    sim.init_from_problem()
    kernel, bx, by = sim.launch()
    assert (bx, by) == (128, 2)
    sim.step(3)
    sim.sync()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = sim.populations()
    assert np.array_equal(f, np.broadcast_to(w[:, None, None], f.shape))   # rest stays rest
    with pytest.raises(vp.VplbmError) as ei:
        sim.set_launch("scalar40", 256, 1)
    assert ei.value.status == 1
    sim.set_launch("scalar40", 32, 8)
    sim.step(2)
    sim.sync()
    sim.close()


def test_penalized_wall_poiseuille_on_the_gpu():
    # The penalized-wall channel of the oracle pin run to its steady state
    # on the GPU: FP64 lands on the oracle's profile, and both FP64 and FP32
    # on the continuum Brinkman solution within the discretisation error the
    # oracle shows at this resolution (3.4e-3 of the peak velocity).
    import math
    import paper_1905_05110_gb300 as vp
    from test_oracle_pins import _brinkman_channel
    p, u, nu = _brinkman_channel(1)
    ny, nx = p["ny"], p["nx"]
    steps = int(12 * ny * ny / (math.pi ** 2 * nu))
    init = (np.ones((ny, nx)), np.tile(u[:, None], (1, nx)), np.zeros((ny, nx)))
    orc = oracle.OracleSim(p, hist_cap=4)
    orc.init_equilibrium(*init)
    orc.step(steps)
    uo = orc.fields()[1].mean(axis=1)
    for precision in ("f64", "f32"):
        sim = vp.Simulation(p, precision=precision, history_capacity=steps + 8)
        sim.init_equilibrium(*init)
        sim.step(steps)
        ug = sim.fields()[1].mean(axis=1)
        if precision == "f64":
            assert np.max(np.abs(ug - uo)) < 1e-10 * np.max(u)
        assert np.max(np.abs(ug - u)) / np.max(u) < 4e-3, precision
        sim.close()
