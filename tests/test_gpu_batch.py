"""Batched sweep: members stepped in one launch per step match the same
simulations stepped alone, and the oracle."""
import numpy as np
import pytest

import oracle
import workloads as wl
from helpers import REC, dev_err, make_pair, moving_bodies, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library(gpu_library):
    return gpu_library


def _members():
    out = []
    for (nx, ny), motion in (((130, 66), "fixed"), ((256, 96), "imposed"), ((194, 70), "free")):
        body = moving_bodies(nx, ny)[motion]
        p = wl.mixed_bc_box(nx, ny, seed=nx, west="velocity", east="zerograd", south="noslip",
                            north="noslip", tau=0.6, body=body)
        p["bc"]["west"] = {"kind": "velocity", "u": (0.04, 0.0)}
        p["init"] = {"rho": 1.0, "u": (0.04, 0.0)}
        out.append(p)
    return out


@pytest.mark.parametrize("precision,tiles_per_block", [("f32", 0), ("f16", 0), ("f64", 0),
                                                     ("f32", 1), ("f32", 8), ("f16", 5), ("f64", 3)])
def test_batch_members_match_standalone_runs(precision, tiles_per_block):
    """Branch mode (0), and tile mode with macro tiles of 1, 3, 5 and 8
    tiles: ragged last macro rows (66, 96 and 70 rows) and the reduction
    tiles of a body spread over several blocks."""
    import paper_1905_05110_gb300 as vp
    probs = _members()
    batch = vp.Batch(probs, precision=precision, history_capacity=256)
    if tiles_per_block == 0:
        batch.set_mode("branches")
        for m in batch.members:
            vp.vplbm_set_launch(m.ctx, vp.KERNELS["scalar48"], 256, 1)
    else:
        batch.set_mode("tiles")
        batch.set_launch(256, 1, tiles_per_block)
        assert batch.launch()[:3] == (256, 1, tiles_per_block)
    batch.init_from_problems()
    batch.step(70)   # two graphs of 32 and 6 single launches
    batch.sync()
    for k, p in enumerate(probs):
        alone = vp.Simulation(p, precision=precision, history_capacity=256)
        alone.set_launch("scalar48", 256, 1)   # the same tile code and budget as the batched kernel
        alone.init_from_problem()
        alone.step(70)
        m = batch.members[k]
        assert m.nstep == 70
        assert dev_err(m.populations(), alone.populations()) < (1e-6 if precision == "f32" else 1e-3)
        hm, ha = m.history(), alone.history()
        assert np.array_equal(hm[:, REC["n_solid"]], ha[:, REC["n_solid"]])
        assert rel_err(hm[:, REC["fy"]], ha[:, REC["fy"]]) < 1e-4
        alone.close()
    assert batch.launch()[3] == 70
    batch.close()


def test_batch_member_matches_oracle():
    import paper_1905_05110_gb300 as vp
    probs = _members()
    batch = vp.Batch(probs, precision="f32", history_capacity=64)
    batch.init_from_problems()
    batch.step(25)
    for k, p in enumerate(probs):
        orc = oracle.OracleSim(p, hist_cap=64)
        shape = (p["ny"], p["nx"])
        orc.init_equilibrium(np.ones(shape), np.full(shape, 0.04), np.zeros(shape))
        orc.step(25)
        assert dev_err(batch.members[k].populations(), orc.populations()) < 1e-4
        hb, ho = batch.members[k].history(), orc.history()
        assert np.array_equal(hb[:, REC["n_solid"]], ho[:, REC["n_solid"]])
    batch.close()


def test_batch_rejects_members_out_of_step_and_autotunes():
    import paper_1905_05110_gb300 as vp
    probs = _members()
    batch = vp.Batch(probs, precision="f32", history_capacity=64)
    batch.init_from_problems()
    vp.vplbm_step(batch.members[1].ctx, 1)
    with pytest.raises(vp.VplbmError) as ei:
        batch.step(1)
    assert ei.value.status == 1
    batch.init_from_problems()
    shape = batch.autotune(4)
    assert shape[0] == "branches" or shape[1:] in ((256, 1, 8), (256, 1, 4), (256, 1, 16), (128, 2, 4),
                                                   (128, 1, 8), (256, 1, 1))
    with pytest.raises(vp.VplbmError):
        batch.set_launch(256, 1, 0)
    with pytest.raises(vp.VplbmError):
        batch.set_launch(96, 1, 1)
    assert batch.launch()[:3] == shape[1:]
    with pytest.raises(vp.VplbmError):
        batch.set_mode(5)
    batch.sync()
    batch.close()


@pytest.mark.parametrize("mode", ["branches", "tiles"])
def test_batch_with_ellipse_and_disk_members(mode):
    """Members of different body shapes in one batch (the tile-mode kernel
    reads the shape per member) match the same simulations stepped alone."""
    import paper_1905_05110_gb300 as vp
    probs = _members()
    e = dict(probs[1]["body"], shape="ellipse", radius_b=0.5 * probs[1]["body"]["radius"], theta=0.4)
    probs[1] = dict(probs[1], body=e)
    batch = vp.Batch(probs, precision="f32", history_capacity=128)
    batch.set_mode(mode)
    if mode == "tiles":
        batch.set_launch(256, 1, 4)
    else:
        for m in batch.members:
            vp.vplbm_set_launch(m.ctx, vp.KERNELS["scalar48"], 256, 1)
    batch.init_from_problems()
    batch.step(40)
    for k, p in enumerate(probs):
        alone = vp.Simulation(p, precision="f32", history_capacity=128)
        alone.set_launch("scalar48", 256, 1)
        alone.init_from_problem()
        alone.step(40)
        m = batch.members[k]
        assert dev_err(m.populations(), alone.populations()) < 1e-6
        assert np.array_equal(m.history()[:, REC["n_solid"]], alone.history()[:, REC["n_solid"]])
        alone.close()
    batch.close()
