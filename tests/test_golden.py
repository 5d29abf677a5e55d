"""The oracle's constants against the values printed in the paper, stored
as text fixtures under tests/golden/ (each file names the equation it
copies).  These are the paper's own numbers, so a transposed row, a wrong
sign or a misplaced velocity in the oracle fails here."""
import os

import numpy as np
import pytest

import oracle
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def test_moment_matrix_is_the_printed_one():
    _, _, M, Minv = oracle.constants()
    printed = _load("mrt_matrix_eq15.txt")
    assert printed.shape == (9, 9)
    assert np.array_equal(M, printed)
    assert np.allclose(Minv @ printed, np.eye(9), atol=1e-15)


def test_velocities_and_weights_are_the_printed_ones():
    c, w, _, _ = oracle.constants()
    t = _load("d2q9_velocities_weights_eq10_eq13.txt")
    assert np.array_equal(t[:, 0], np.arange(9))
    assert np.array_equal(c, t[:, 1:3].astype(int))
    assert np.array_equal(w * 36.0, t[:, 3])


@pytest.mark.parametrize("seed", range(4))
def test_moment_equilibria_are_the_printed_ones(seed):
    # Eq. (14) as printed, through the coefficient table, against both the
    # oracle's moment equilibria and M applied to its Eq. (11) equilibrium.
    rng = np.random.default_rng(100 + seed)
    coef = _load("moment_equilibria_eq14.txt")
    _, _, M, _ = oracle.constants()
    for _ in range(8):
        rho = 1.0 + rng.uniform(-0.2, 0.2)
        ux, uy = rng.uniform(-0.15, 0.15, size=2)
        mono = np.array([1.0, ux * ux + uy * uy, ux, uy, ux * ux - uy * uy, ux * uy])
        printed = rho * (coef @ mono)
        assert np.allclose(oracle.moment_equilibrium(rho, ux, uy), printed, rtol=0, atol=1e-15)
        assert np.allclose(M @ oracle.equilibrium(rho, ux, uy), printed, rtol=0, atol=1e-15)


@pytest.mark.parametrize("tau", [0.56, 0.6, 0.8, 1.3])
def test_paper_rates_are_the_printed_ones(tau):
    t = _load("relaxation_rates_sec3.txt")
    expect = np.where(np.isnan(t[:, 1]), 1.0 / tau, t[:, 1])
    assert np.array_equal(np.asarray(wl.paper_rates(tau)), expect)


# ---- oracle regression fixtures (written by tests/golden/make_oracle_golden.py) ----

def _generator():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_oracle_golden", os.path.join(GOLDEN, "make_oracle_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


GEN = _generator()


def _scaled_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("case", list(GEN.CASES))
def test_oracle_reproduces_its_regression_fixture(case):
    # The stored records and populations of each small problem: any change to
    # the oracle's arithmetic shows here (tolerance: the libm differences of
    # another host's sin / cos / sqrt, far below any change of a term).
    hist, idx, vals = GEN.run_case(case)
    ph, pp = GEN.paths(case)
    h0 = np.loadtxt(ph)
    p0 = np.loadtxt(pp)
    assert h0.shape == hist.shape
    ns = GEN.HISTORY_FIELDS.index("n_solid")
    assert np.array_equal(hist[:, ns], h0[:, ns])
    for k, name in enumerate(GEN.HISTORY_FIELDS):
        if name != "n_solid":
            assert _scaled_err(hist[:, k], h0[:, k]) < 1e-11, name
    assert np.array_equal(idx, p0[:, :3].astype(int))
    assert np.allclose(vals, p0[:, 3], rtol=1e-12, atol=1e-15)
