"""Host fields in and out of a simulation: page-locked (pinned) arrays are
read and written in place by the kernels, pageable ones go through device
memory; both routes must give the same state and the same fields."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library(gpu_library):
    return gpu_library


@pytest.mark.parametrize("precision", ["f64", "f32", "f16"])
def test_pinned_and_pageable_fields_give_the_same_state_and_fields(precision):
    import torch
    import paper_1905_05110_gb300 as vp
    p = wl.oscillating_disk(nx=300, ny=130, diameter=20.0, x_c=61.3)
    ny, nx = p["ny"], p["nx"]
    rng = np.random.default_rng(3)
    host = [1.0 + 0.01 * rng.standard_normal((ny, nx)), 0.04 + 0.01 * rng.standard_normal((ny, nx)),
            0.01 * rng.standard_normal((ny, nx))]
    pinned = [torch.empty((ny, nx), dtype=torch.float64, pin_memory=True) for _ in range(6)]
    for t, a in zip(pinned, host):
        t.copy_(torch.from_numpy(a))
    sims = []
    for fields in ([h.copy() for h in host], [t.numpy() for t in pinned[:3]]):
        s = vp.Simulation(p, precision=precision, history_capacity=64)
        vp.vplbm_init_equilibrium(s.ctx, *fields)
        s.step(9)
        sims.append(s)
    assert np.array_equal(sims[0].populations(), sims[1].populations())
    out_pageable = [np.empty((ny, nx)) for _ in range(3)]
    vp.vplbm_get_fields(sims[1].ctx, *out_pageable)
    out_pinned = [t.numpy() for t in pinned[3:]]
    for t in pinned[3:]:
        t.fill_(np.nan)
    vp.vplbm_get_fields(sims[1].ctx, *out_pinned)
    for a, b in zip(out_pageable, out_pinned):
        assert np.array_equal(a, b)
    # one pinned output with NULL others: written in place, the others untouched
    pinned[3].fill_(np.nan)
    vp.vplbm_get_fields(sims[1].ctx, None, pinned[3].numpy(), None)
    assert np.array_equal(pinned[3].numpy(), out_pageable[1])
    for s in sims:
        s.close()
