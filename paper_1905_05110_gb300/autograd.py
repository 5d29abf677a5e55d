"""The discrete adjoint behind ``torch.autograd``.

``adjoint_objectives(u_in, eta, s_nu, s_e, problem, nsteps, window_start)``
returns the tensor (J1, J2) = (mean C_D, RMS C_L) over the steps
[window_start, nsteps) of a run of the problem from its initial state, with
the parameters set to the given tensors: the west wall's inlet u_x profile
(one value per inlet node), eta (Eq. 2), s_nu (= s_7 = s_8, Eq. 16) and s_e
(= s_1).  Its backward pass is one run of ``vplbm_adjoint`` with the
weights (w_cd, w_cl) = the incoming gradient, since the adjoint of the
weighted objective w_cd J1 + w_cl J2 gives exactly that vector-Jacobian
product.  The body must move on a prescribed path (chi is the binary mask of
each step), as the adjoint requires.  Forward and backward both run on the
GPU through the C ABI; nothing here computes a step of the method.
"""
from __future__ import annotations

import numpy as np

from . import Simulation

__all__ = ["AdjointObjectives", "adjoint_objectives", "problem_with_params"]

_CD, _CL = 4, 5   # columns of C_D and C_L in a history record


def problem_with_params(problem: dict, u_in, eta, s_nu, s_e) -> dict:
    """Copy of a problem with the adjoint's four parameter groups replaced."""
    p = dict(problem)
    p["s"] = list(problem["s"])
    p["bc"] = {k: dict(v) for k, v in problem["bc"].items()}
    p["bc"]["west"]["ux_profile"] = np.asarray(u_in, dtype=np.float64).copy()
    p["eta"] = float(eta)
    p["s"][7] = p["s"][8] = float(s_nu)
    p["s"][1] = float(s_e)
    return p


def _run_objectives(p: dict, nsteps: int, window_start: int, precision: str) -> tuple:
    sim = Simulation(p, precision=precision, history_capacity=nsteps)
    try:
        sim.init_from_problem()
        sim.step(nsteps)
        h = sim.history(0, nsteps)
    finally:
        sim.close()
    w = h[window_start:]
    return float(w[:, _CD].mean()), float(np.sqrt((w[:, _CL] ** 2).mean()))


class AdjointObjectives:
    """Namespace of the torch.autograd.Function (built on first use so that
    importing this module does not import torch)."""

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            import torch

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, u_in, eta, s_nu, s_e, problem, nsteps, window_start, precision,
                            checkpoint_interval):
                    vals = [t.detach().cpu().double() for t in (u_in, eta, s_nu, s_e)]
                    p = problem_with_params(problem, vals[0].numpy(), vals[1].item(), vals[2].item(),
                                            vals[3].item())
                    ctx.p = p
                    ctx.args = (int(nsteps), int(window_start), precision, int(checkpoint_interval))
                    ctx.like = (u_in, eta, s_nu, s_e)
                    j1, j2 = _run_objectives(p, int(nsteps), int(window_start), precision)
                    return torch.tensor([j1, j2], dtype=torch.float64, device=u_in.device)

                @staticmethod
                def backward(ctx, g):
                    nsteps, window_start, precision, ckpt = ctx.args
                    gw = g.detach().cpu().double().numpy()
                    sim = Simulation(ctx.p, precision=precision, history_capacity=nsteps)
                    try:
                        sim.init_from_problem()
                        grad, _ = sim.adjoint(nsteps, window_start, float(gw[0]), float(gw[1]),
                                              checkpoint_interval=ckpt)
                    finally:
                        sim.close()
                    ny = len(grad) - 3
                    u_in, eta, s_nu, s_e = ctx.like
                    out = [torch.as_tensor(grad[:ny], dtype=u_in.dtype, device=u_in.device)]
                    for t, k in ((eta, ny), (s_nu, ny + 1), (s_e, ny + 2)):
                        out.append(torch.as_tensor(grad[k], dtype=t.dtype, device=t.device).reshape(t.shape))
                    return (*out, None, None, None, None, None)

            cls._fn = _Fn
        return cls._fn


def adjoint_objectives(u_in, eta, s_nu, s_e, problem: dict, nsteps: int, window_start: int,
                       precision: str = "f64", checkpoint_interval: int = 0):
    """(mean C_D, RMS C_L) of the run, differentiable in the four parameter
    tensors (u_in: [ny]; eta, s_nu, s_e: scalars) through the discrete
    adjoint.  precision: "f64" (FP64 adjoint) or "f32" (FP32 adjoint with
    FP64 parameter sums)."""
    return AdjointObjectives.function().apply(u_in, eta, s_nu, s_e, problem, nsteps, window_start, precision,
                                              checkpoint_interval)
