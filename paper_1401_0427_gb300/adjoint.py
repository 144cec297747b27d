"""Gradients of the 2D scheme through time for PyTorch: a torch.autograd.Function whose
forward runs T fused steps from an equilibrium start at rest, f = f^eq(h0, 0, 0), and
whose backward runs the discrete adjoint with sqrt(T) checkpointing (lbm_sw_adjoint).

Only device memory and streams come from PyTorch; every step, replay and adjoint
step runs in the CUDA library.
"""

from __future__ import annotations

import torch

from . import lbm_sw


class ShallowWaterRun(torch.autograd.Function):
    """h_T = run(h0): depth after `steps` steps from rest (discharge zero).

    The forward pass runs on the caller's Simulation: it overwrites that handle's state
    (set_state(h0, 0, 0), then `steps` steps), so afterwards `sim` holds the state at step T.
    Its checkpoint tape owns its own device memory and is released when the autograd graph
    that holds it is freed, so backward may run more than once (retain_graph=True); each
    backward replays the tape's checkpoints and leaves the handle's state alone."""

    @staticmethod
    def forward(ctx, h0: torch.Tensor, sim: lbm_sw.Simulation, steps: int, interval: int = 0):
        assert h0.is_cuda and h0.dtype == torch.float64 and h0.is_contiguous()
        zero = torch.zeros_like(h0)
        sim.set_state(h0, zero, zero)
        tape = lbm_sw.Tape(sim, steps, interval)
        tape.record()
        hT = torch.empty_like(h0)
        huT = torch.empty_like(h0)
        hvT = torch.empty_like(h0)
        sim.moments_into(hT, huT, hvT)
        ctx.tape = tape
        return hT

    @staticmethod
    def backward(ctx, g_hT: torch.Tensor):
        g = g_hT.contiguous().to(torch.float64)
        d_h0 = ctx.tape.adjoint(g)
        return d_h0, None, None, None


def run(h0: torch.Tensor, sim: lbm_sw.Simulation, steps: int, interval: int = 0) -> torch.Tensor:
    return ShallowWaterRun.apply(h0, sim, steps, interval)


def recover_initial_depth(h_obs: torch.Tensor, sim: lbm_sw.Simulation, steps: int, h_guess: torch.Tensor,
                          iterations: int = 20, interval: int = 0):
    """Fit h0 so that run(h0) matches h_obs in least squares (L = 1/2 sum (h_T - h_obs)^2)
    with L-BFGS; returns (h0, list of losses)."""
    h0 = h_guess.clone().requires_grad_(True)
    opt = torch.optim.LBFGS([h0], lr=1.0, max_iter=iterations, history_size=10, line_search_fn="strong_wolfe")
    losses = []

    def closure():
        opt.zero_grad()
        loss = 0.5 * ((run(h0, sim, steps, interval) - h_obs) ** 2).sum()
        loss.backward()
        losses.append(float(loss.detach()))
        return loss

    opt.step(closure)
    return h0.detach(), losses
