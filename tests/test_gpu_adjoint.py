"""GPU discrete adjoint against the FP64 oracle adjoint (itself pinned by
central finite differences in the CPU suite)."""
import numpy as np
import pytest

import oracle
import workloads as wl
from helpers import dev_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library(gpu_library):
    return gpu_library


def _init_both(p, precision, hist=512):
    import paper_1905_05110_gb300 as vp
    g = vp.Simulation(p, precision=precision, history_capacity=hist)
    g.init_from_problem()
    o = oracle.OracleSim(p, hist_cap=hist)
    sh = (p["ny"], p["nx"])
    u = p["init"]["u"]
    o.init_equilibrium(np.ones(sh), np.full(sh, u[0]), np.full(sh, u[1]))
    return g, o


def _cases():
    base = wl.adjoint_channel()
    yield "channel", base
    for south, north in (("periodic", "periodic"), ("noslip", "velocity")):
        p = wl.mixed_bc_box(26, 15, seed=4, west="velocity", east="zerograd", south=south, north=north, tau=0.62,
                            body=dict(base["body"], x=9.0, y=7.4))
        p["bc"]["west"] = dict(base["bc"]["west"])
        p["bc"]["west"]["ux_profile"] = wl.parabolic_profile(15, 0.03)
        p["init"] = {"rho": 1.0, "u": (0.03, 0.0)}
        p["eta"] = 0.05
        yield f"box_{south}_{north}", p


@pytest.mark.parametrize("ckpt", [0, 7, 1])
@pytest.mark.parametrize("weights", [(1.0, 0.0), (0.0, 1.0)])
@pytest.mark.parametrize("case", ["channel", "box_periodic_periodic", "box_noslip_velocity"])
def test_fp64_adjoint_matches_oracle(case, weights, ckpt):
    p = dict(_cases())[case]
    N, w0 = 30, 15
    g, o = _init_both(p, "f64")
    gg, gj = g.adjoint(N, w0, *weights, checkpoint_interval=ckpt)
    og, oj = o.adjoint(N, w0, *weights)
    assert np.allclose(gj, oj, rtol=1e-11)
    scale_u = np.max(np.abs(og[:-3]))
    assert np.max(np.abs(gg[:-3] - og[:-3])) < 1e-9 * scale_u
    for k in (-3, -2, -1):
        assert abs(gg[k] - og[k]) < 1e-9 * abs(og[k]), k
    # the context ends at the state after the forward run
    assert g.nstep == N
    assert dev_err(g.populations(), o.populations()) < 1e-12


@pytest.mark.parametrize("weights", [(1.0, 0.0), (0.0, 1.0)])
def test_fp32_adjoint_close_to_oracle(weights):
    p = wl.adjoint_channel()
    N, w0 = 30, 15
    g, o = _init_both(p, "f32")
    gg, gj = g.adjoint(N, w0, *weights)
    og, oj = o.adjoint(N, w0, *weights)
    assert np.allclose(gj, oj, rtol=1e-4)
    scale_u = np.max(np.abs(og[:-3]))
    assert np.max(np.abs(gg[:-3] - og[:-3])) < 1e-3 * scale_u
    for k in (-3, -2, -1):
        assert abs(gg[k] - og[k]) < 1e-3 * abs(og[k]), k


@pytest.mark.parametrize("nx", [72, 70])
@pytest.mark.parametrize("weights", [(1.0, 0.0), (0.0, 1.0)])
def test_fp32_adjoint_multi_tile_close_to_oracle(nx, weights):
    """A lattice of several reverse-kernel tiles in x and y, with ragged last
    tiles (interior tiles 32 x 16 nodes), against the FP64 oracle adjoint."""
    p = wl.adjoint_channel(nx=nx, ny=40, radius=6.0)
    N, w0 = 30, 15
    g, o = _init_both(p, "f32")
    gg, gj = g.adjoint(N, w0, *weights, checkpoint_interval=7)
    og, oj = o.adjoint(N, w0, *weights)
    assert np.allclose(gj, oj, rtol=1e-4)
    scale_u = np.max(np.abs(og[:-3]))
    assert np.max(np.abs(gg[:-3] - og[:-3])) < 1e-3 * scale_u
    for k in (-3, -2, -1):
        assert abs(gg[k] - og[k]) < 1e-3 * abs(og[k]), k
    # a second run repeats the gradient bit for bit
    g2, _ = _init_both(p, "f32")
    gg2, _ = g2.adjoint(N, w0, *weights, checkpoint_interval=7)
    assert np.array_equal(gg, gg2)


@pytest.mark.parametrize("ckpt", [0, 13])
def test_fp64_adjoint_long_run_matches_oracle(ckpt):
    """A 64 x 32 channel over 200 steps (several checkpoint segments, the
    oscillating disk crossing nodes many times) against the FP64 oracle
    adjoint."""
    p = wl.adjoint_channel(nx=64, ny=32, radius=5.0, steps=200)
    N, w0 = 200, 100
    g, o = _init_both(p, "f64", hist=N + 8)
    gg, gj = g.adjoint(N, w0, 1.0, 1.0, checkpoint_interval=ckpt)
    og, oj = o.adjoint(N, w0, 1.0, 1.0)
    assert np.allclose(gj, oj, rtol=1e-11)
    scale_u = np.max(np.abs(og[:-3]))
    assert np.max(np.abs(gg[:-3] - og[:-3])) < 1e-9 * scale_u
    for k in (-3, -2, -1):
        assert abs(gg[k] - og[k]) < 1e-9 * abs(og[k]), k


def test_adjoint_workspace_kept_between_calls():
    """The context keeps the adjoint's device workspace: a repeated call, a
    call that needs a larger workspace (more checkpoints and a longer
    segment) and a smaller call after it give, bit for bit, what a fresh
    context gives."""
    import paper_1905_05110_gb300 as vp
    p = wl.adjoint_channel(nx=72, ny=40, radius=6.0)

    def run(sim, n, k):
        sim.init_from_problem()
        return sim.adjoint(n, n // 2, 1.0, 1.0, checkpoint_interval=k)

    g = vp.Simulation(p, precision="f32", history_capacity=128)
    a1, ja1 = run(g, 30, 7)
    a2, ja2 = run(g, 30, 7)
    assert np.array_equal(a1, a2) and np.array_equal(ja1, ja2)
    b1, jb1 = run(g, 60, 5)   # 12 checkpoints and 2 x 5 store slots: the workspace grows
    c1, _ = run(g, 30, 7)     # fits the grown workspace
    assert np.array_equal(c1, a1)
    fresh = vp.Simulation(p, precision="f32", history_capacity=128)
    b2, jb2 = run(fresh, 60, 5)
    assert np.array_equal(b1, b2) and np.array_equal(jb1, jb2)
    g.close()
    fresh.close()


def test_adjoint_rejects_free_bodies():
    import paper_1905_05110_gb300 as vp
    p = wl.sedimenting_disk(nx=64, ny=128, diameter=8)
    g = vp.Simulation(p, precision="f64", history_capacity=64)
    g.init_from_problem()
    with pytest.raises(vp.VplbmError) as ei:
        g.adjoint(10, 5)
    assert ei.value.status == 6


def _objective_gpu(p, N, w0):
    import paper_1905_05110_gb300 as vp
    g = vp.Simulation(p, precision="f64", history_capacity=N + 8)
    g.init_from_problem()
    g.step(N)
    h = g.history(0, N)
    g.close()
    return h[w0:, 4].mean() + np.sqrt(np.mean(h[w0:, 5] ** 2))


def test_adjoint_directional_derivatives_match_central_differences():
    # The oscillating-disk gradient workload, scaled down: 8 random directions
    # in the 99-dimensional parameter space (inlet profile, eta, s_nu, s_e),
    # central differences with h = 1e-4 of each parameter's scale, FP64.
    p = wl.adjoint_disk(nx=192, ny=96, diameter=12, steps=400, checkpoint_interval=20)
    p["eta"] = 0.02
    N, w0 = 400, 200
    import paper_1905_05110_gb300 as vp
    g = vp.Simulation(p, precision="f64", history_capacity=N + 8)
    g.init_from_problem()
    grad, js = g.adjoint(N, w0, 1.0, 1.0, checkpoint_interval=20)
    prof = p["bc"]["west"]["ux_profile"]
    scale = np.concatenate([np.full(p["ny"], 0.04), [p["eta"], p["s"][7], p["s"][1]]])
    rng = np.random.default_rng(5)
    h = 1e-4
    for _ in range(8):
        v = rng.standard_normal(p["ny"] + 3)
        v /= np.linalg.norm(v)
        dth = h * scale * v

        def perturbed(sign):
            return wl.with_params(p, u_in_profile=prof + sign * dth[:-3], eta=p["eta"] + sign * dth[-3],
                                  s_nu=p["s"][7] + sign * dth[-2], s_e=p["s"][1] + sign * dth[-1])

        fd = (_objective_gpu(perturbed(1), N, w0) - _objective_gpu(perturbed(-1), N, w0)) / (2 * h)
        adj = float(grad @ (scale * v))
        assert abs(fd - adj) < 1e-4 * abs(adj) + 1e-10, (fd, adj)


def test_autograd_function_gives_the_adjoint_gradient_and_passes_gradcheck():
    # The torch.autograd.Function: the forward's (J1, J2) equal the
    # adjoint's, the backward of g . J is the adjoint run with weights g, and
    # torch's own gradcheck (central differences of the forward through the
    # C ABI, FP64) accepts it.
    import torch
    from paper_1905_05110_gb300.autograd import adjoint_objectives
    p = wl.adjoint_channel()
    N, w0 = 30, 15
    dev = torch.device("cuda")
    u = torch.tensor(p["bc"]["west"]["ux_profile"], dtype=torch.float64, device=dev, requires_grad=True)
    eta = torch.tensor(p["eta"], dtype=torch.float64, device=dev, requires_grad=True)
    s_nu = torch.tensor(p["s"][7], dtype=torch.float64, device=dev, requires_grad=True)
    s_e = torch.tensor(p["s"][1], dtype=torch.float64, device=dev, requires_grad=True)
    J = adjoint_objectives(u, eta, s_nu, s_e, p, N, w0)
    g, o = _init_both(p, "f64")
    grad, js = g.adjoint(N, w0, 0.7, 0.3)
    assert np.allclose(J.detach().cpu().numpy(), js, rtol=1e-13)
    (0.7 * J[0] + 0.3 * J[1]).backward()
    got = np.concatenate([u.grad.cpu().numpy(), [eta.grad.item(), s_nu.grad.item(), s_e.grad.item()]])
    assert np.array_equal(got, grad)

    def f(u_, eta_, s_nu_, s_e_):
        return adjoint_objectives(u_, eta_, s_nu_, s_e_, p, N, w0)

    args = tuple(t.detach().clone().requires_grad_(True) for t in (u, eta, s_nu, s_e))
    assert torch.autograd.gradcheck(f, args, eps=1e-6, atol=1e-7, rtol=1e-4)
