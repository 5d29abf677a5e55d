"""The CUDA path through the C ABI against the stored oracle regression
fixtures of tests/golden (written by make_oracle_golden.py from the FP64
oracle alone): records and sampled populations of four small problems
(an imposed disk among every wall kind, a free spring-mounted disk in a
periodic box from random populations, the paper's channel with its
convective outlet, a pitching ellipse under BGK collision)."""
import importlib.util
import os

import numpy as np
import pytest

from helpers import REC, rel_err

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_spec = importlib.util.spec_from_file_location("make_oracle_golden", os.path.join(GOLDEN, "make_oracle_golden.py"))
GEN = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(GEN)

# FP64: rounding-order differences only; FP32 storage: 1e-4 of a population
# deviation of 0.05 (the bound the live-oracle parity tests apply)
FORCE_TOL = {"f64": 1e-10, "f32": 1e-3}
POP_TOL = {"f64": 1e-13, "f32": 5e-6}


@pytest.fixture(scope="module", autouse=True)
def _library(gpu_library):
    return gpu_library


@pytest.mark.parametrize("case", list(GEN.CASES))
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_gpu_matches_stored_oracle_fixture(case, precision):
    import paper_1905_05110_gb300 as vp
    p, f0, steps = GEN.CASES[case]()
    if precision == "f32" and (p.get("body") or {}).get("motion") == "free":
        pytest.skip("a free body's FP32 trajectory is compared with the live oracle in test_gpu_parity")
    sim = vp.Simulation(p, precision=precision, history_capacity=steps + 8)
    if f0 is not None:
        sim.set_populations(f0)
    else:
        sim.init_from_problem()
    sim.step(steps)
    h = sim.history(0, steps)
    f = sim.populations()
    sim.close()
    h0 = np.loadtxt(GEN.paths(case)[0])
    p0 = np.loadtxt(GEN.paths(case)[1])
    cols = {name: k for k, name in enumerate(GEN.HISTORY_FIELDS)}
    assert np.array_equal(h[:, REC["n_solid"]], h0[:, cols["n_solid"]])
    for key in ("fx", "fy", "torque", "fpen_x", "fpen_y", "tpen"):
        assert rel_err(h[:, REC[key]], h0[:, cols[key]]) < FORCE_TOL[precision], key
    for key in ("x", "y", "theta", "vx", "vy", "omega"):
        assert rel_err(h[:, REC[key]], h0[:, cols[key]]) < FORCE_TOL[precision], key
    idx = p0[:, :3].astype(int)
    assert np.allclose(f[idx[:, 0], idx[:, 1], idx[:, 2]], p0[:, 3], rtol=0, atol=POP_TOL[precision])
