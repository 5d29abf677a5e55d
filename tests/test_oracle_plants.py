"""The pins bind the oracle: each of these plausible mistakes, planted in
the oracle at compile time (ORACLE_PLANT=k), makes the paper-based pins of
test_oracle_pins.py and test_golden.py fail (the regression fixtures are
left out, since they would catch any change at all)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PLANTS = {
    1: "the sign of q_x in the moment equilibria (Eq. 14)",
    2: "the (c.u) c term of the Guo forcing (Eq. 12) dropped",
    3: "the diagonal weights 1/18 instead of 1/36 (Eq. 13)",
    4: "the 1/2 of the eta-stable penalized velocity (Eq. 22) dropped",
    5: "RK4 reduced to forward Euler",
    6: "the sign of the momentum-exchange torque (Eq. 27)",
    7: "the sign of the moving-wall term of the bounce-back",
    8: "the outlet's source row j instead of j - c_ay (zero-gradient and convective rules)",
    9: "the adjoint: a solid node's own momentum-exchange term (Eqs. 25-27) dropped from L_n",
    10: "the adjoint: the forcing factor (1 - s_r/2) of Eq. 17 taken as (1 - s_r)",
    11: "the adjoint: the sign of the inlet-profile gradient",
    12: "the BGK forcing prefactor (1 - 1/(2 tau)) of Eq. 12 dropped",
    13: "a symmetry wall that bounces populations back instead of mirroring them",
    14: "the ellipse's semi-axes swapped in its predicate",
    15: "the rectangle's body frame turned by -theta instead of theta",
    16: "the sign of the penalization reaction on the body",
    17: "the momentum exchange without the node's own streamed-in momentum (Eq. 25)",
    18: "the convective outlet's two weights swapped (f_prev and the upwind value)",
    19: "the imposed motion's velocity taken as the sine instead of the cosine",
}


@pytest.mark.parametrize("k", sorted(PLANTS))
def test_pins_catch_planted_mistake(k):
    env = dict(os.environ, VPLBM_ORACLE_PLANT=str(k))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "-k", "not regression", "tests/test_oracle_pins.py", "tests/test_golden.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    # exit status 1: tests ran and one failed (not a collection or build error)
    assert r.returncode == 1, f"plant {k} ({PLANTS[k]}) not caught:\n{r.stdout[-3000:]}\n{r.stderr[-2000:]}"
    failed = [line for line in r.stdout.splitlines() if line.startswith("FAILED")]
    assert failed, r.stdout[-2000:]
