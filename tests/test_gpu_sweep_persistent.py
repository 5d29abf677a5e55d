"""Persistent sweep: every member of a batch advanced over many steps by one
cooperative launch (a work queue of body tiles and node-pair tiles, a
grid-wide barrier per step).

Each work item runs the tile code of the one-lattice kernels, so a member's
populations, history records and body state must equal, bit for bit, those
of the same simulation stepped alone with the node-pair kernel (one-node
kernel for an odd nx) at the same block shape: the body tiles, and with
them the order of the force sums, are the same.  Members cover the three
motion kinds, an odd nx (one-node tiles), a convective outlet (its outlet
column is written in one step and read in the next, inside the launch) and
ragged tile edges."""
import numpy as np
import pytest

import oracle
import workloads as wl
from helpers import REC, dev_err, moving_bodies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library(gpu_library):
    return gpu_library


def _members(ellipse=False):
    out = []
    for (nx, ny), motion, east in (((130, 66), "fixed", "zerograd"), ((256, 96), "imposed", "zerograd"),
                                   ((194, 70), "free", "zerograd"), ((131, 50), "free", "convective")):
        body = moving_bodies(nx, ny)[motion]
        p = wl.mixed_bc_box(nx, ny, seed=nx, west="velocity", east="zerograd", south="noslip",
                            north="noslip", tau=0.6, body=body)
        p["bc"]["west"] = {"kind": "velocity", "u": (0.04, 0.0)}
        if east == "convective":
            p["bc"]["east"] = {"kind": "convective", "u": (0.04, 0.0)}
        p["init"] = {"rho": 1.0, "u": (0.04, 0.0)}
        out.append(p)
    if ellipse:
        e = dict(out[1]["body"], shape="ellipse", radius_b=0.5 * out[1]["body"]["radius"], theta=0.4)
        out[1] = dict(out[1], body=e)
    return out


def _alone(p, precision, bx, by, nsteps, cap):
    import paper_1905_05110_gb300 as vp
    s = vp.Simulation(p, precision=precision, history_capacity=cap)
    s.set_launch("pair" if p["nx"] % 2 == 0 else "scalar48", bx, by)
    s.init_from_problem()
    s.step(nsteps)
    return s


def _check_members(batch, probs, precision, bx, by, nsteps, cap):
    for k, p in enumerate(probs):
        alone = _alone(p, precision, bx, by, nsteps, cap)
        m = batch.members[k]
        assert m.nstep == nsteps
        assert np.array_equal(m.populations(), alone.populations()), (k, p["nx"], p["ny"])
        first = max(0, nsteps - cap)
        assert np.array_equal(m.history(first, nsteps - first), alone.history(first, nsteps - first)), k
        qa, va = alone.body_state()
        qm, vm = m.body_state()
        assert np.array_equal(qm, qa) and np.array_equal(vm, va), k
        alone.close()


@pytest.mark.parametrize("precision,shape", [("f32", (64, 4, 2, False)), ("f16", (64, 4, 2, False)),
                                             ("f32", (32, 8, 1, True)), ("f32", (128, 2, 3, False)),
                                             ("f16", (256, 1, 16, True))])
def test_persistent_members_equal_standalone_runs_bitwise(precision, shape):
    """70 steps in one launch; chunks of 1, 2, 3 (padded steps) and 16
    items; parameters in shared or device memory."""
    import paper_1905_05110_gb300 as vp
    probs = _members()
    bx, by, chunk, psmem = shape
    batch = vp.Batch(probs, precision=precision, history_capacity=256)
    batch.set_persistent(bx, by, chunk, psmem)
    batch.set_mode("persistent")
    assert batch.persistent()[:4] == (bx, by, chunk, int(psmem))
    assert batch.persistent()[4] > 0
    batch.init_from_problems()
    batch.step(70)
    batch.sync()
    assert batch.persistent()[5] == 1
    _check_members(batch, probs, precision, bx, by, 70, 256)
    batch.close()


def test_persistent_graph_and_odd_start():
    """A 1024-step graph of one cooperative launch from an even step, then
    direct launches from an odd step."""
    import paper_1905_05110_gb300 as vp
    probs = _members()
    batch = vp.Batch(probs, precision="f32", history_capacity=512)
    batch.set_persistent(64, 4, 2, False)
    batch.set_mode("persistent")
    batch.init_from_problems()
    batch.step(1024)
    batch.step(3)
    batch.step(1030)
    batch.sync()
    assert batch.persistent()[5] == 4
    _check_members(batch, probs, "f32", 64, 4, 2057, 512)
    batch.close()


def test_persistent_ellipse_member():
    """A member of another body shape: the kernel instantiation for any shape."""
    import paper_1905_05110_gb300 as vp
    probs = _members(ellipse=True)
    batch = vp.Batch(probs, precision="f32", history_capacity=64)
    batch.set_mode("persistent")
    batch.init_from_problems()
    batch.step(40)
    batch.sync()
    bx, by = batch.persistent()[:2]
    _check_members(batch, probs, "f32", bx, by, 40, 64)
    batch.close()


def test_persistent_matches_oracle():
    import paper_1905_05110_gb300 as vp
    probs = _members()
    batch = vp.Batch(probs, precision="f32", history_capacity=64)
    batch.set_mode("persistent")
    batch.init_from_problems()
    batch.step(25)
    batch.sync()
    for k, p in enumerate(probs):
        orc = oracle.OracleSim(p, hist_cap=64)
        shape = (p["ny"], p["nx"])
        orc.init_equilibrium(np.ones(shape), np.full(shape, 0.04), np.zeros(shape))
        orc.step(25)
        assert dev_err(batch.members[k].populations(), orc.populations()) < 1e-4
        hb, ho = batch.members[k].history(), orc.history()
        assert np.array_equal(hb[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    batch.close()


def test_persistent_barrier_timeout_is_reported_and_the_batch_recovers():
    """Every barrier waits for one arrival more than the grid makes: the
    wait gives up after 20 ms, the launch's blocks leave, and the next sync
    reports VPLBM_ETIMEOUT once.  With the hook off, the re-initialised
    batch runs on and matches the standalone runs."""
    import paper_1905_05110_gb300 as vp
    probs = _members()
    batch = vp.Batch(probs, precision="f32", history_capacity=64)
    batch.set_persistent(64, 4, 2, False)
    batch.set_mode("persistent")
    batch.init_from_problems()
    batch.inject_barrier_timeout(True)
    batch.step(6)
    with pytest.raises(vp.VplbmError) as ei:
        batch.sync()
    assert ei.value.status == 5 and "barrier" in str(ei.value)
    batch.sync()   # reported once
    batch.inject_barrier_timeout(False)
    batch.init_from_problems()   # step 0 again, tickets and error words cleared
    batch.step(30)
    batch.sync()
    _check_members(batch, probs, "f32", 64, 4, 30, 64)
    batch.close()


def test_persistent_refusals():
    import paper_1905_05110_gb300 as vp
    probs = _members()[:2]
    b64 = vp.Batch(probs, precision="f64", history_capacity=16)
    with pytest.raises(vp.VplbmError) as ei:
        b64.set_mode("persistent")
    assert ei.value.status == 6
    with pytest.raises(vp.VplbmError) as ei:
        b64.set_persistent(64, 4, 2, False)
    assert ei.value.status == 6
    b64.close()
    b = vp.Batch(probs, precision="f32", history_capacity=16)
    for bad in ((64, 2, 2, False), (48, 4, 2, False), (64, 4, 0, False), (64, 4, 17, False)):
        with pytest.raises(vp.VplbmError) as ei:
            b.set_persistent(*bad)
        assert ei.value.status == 1
    assert b.persistent()[:4] == (32, 8, 4, 1)
    b.close()
