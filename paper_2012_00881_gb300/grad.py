"""Differentiable form: the witness energy gain as a torch.autograd.Function.

forward(theta, table): the driver bunch from its eight parameters on fixed
normals (qs_bigaussian_beam), the plasma lattice with the radial density
table (qs_init_plasma), one 3D step with every bunch depositing
(qs_step3d) and the mean energy gain of the witness over one push of dt
(qs_beam_gain).  backward: the cotangent of the stored wake from the gain
(qs_beam_gain), the reverse slice loop (qs_step3d_adjoint), then the chain
rules of the bunch deposit (qs_beam_deposit_adjoint), of the bunch
parameters (qs_bigaussian_adjoint) and of the density table
(qs_profile_adjoint).  Every step runs in libqs; this module only calls it.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import _binding as B


class _Problem:
    """What the loss holds fixed: the context, the driver's normals and
    Lorentz factor, the witness, dt and the profile's radius."""

    def __init__(self, ctx: "B.Context", z, gamma: float, witness: "B.Beam", dt: float,
                 ppc: int, r_max: float, checkpoint_every: int = 0, schedule=None):
        self.ctx = ctx
        self.z = z
        self.gamma = float(gamma)
        self.witness = witness
        self.dt = float(dt)
        self.ppc = int(ppc)
        self.r_max = float(r_max)
        self.checkpoint_every = int(checkpoint_every)
        # sub-step counts per base interval held fixed (None: the adaptive rule)
        self.schedule = None if schedule is None else [int(v) for v in schedule]


class WitnessGain(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, table, prob: _Problem):
        th = theta.detach().cpu().double().tolist()
        tb = table.detach().cpu().double().tolist()
        c = prob.ctx
        c.init_plasma(prob.ppc, tb, prob.r_max)
        drv = B.bigaussian_beam(th, prob.z, prob.gamma)
        c.step3d([drv, prob.witness], schedule=prob.schedule)
        gain = c.beam_gain(prob.witness, prob.dt)
        fctx.prob = prob
        fctx.th = th
        fctx.n_coef = len(tb)
        fctx.drv = drv
        return torch.tensor(gain, dtype=torch.float64)

    @staticmethod
    def backward(fctx, g):
        prob = fctx.prob
        c = prob.ctx
        d_hist = torch.zeros((5, c.n_xi, c.n, c.n), dtype=torch.float64, device="cuda")
        c.beam_gain(prob.witness, prob.dt, d_hist)
        d_jzb, d_w, d_nion, _ = c.step3d_adjoint(d_hist, prob.checkpoint_every)
        dx, dy, dxi, dw = c.beam_deposit_adjoint(fctx.drv, d_jzb)
        d_theta = B.bigaussian_adjoint(fctx.th, prob.z, dx, dy, dxi, dw)
        d_table = c.profile_adjoint(d_w, d_nion, fctx.n_coef, prob.r_max)
        gv = float(g)
        return (torch.tensor(d_theta * gv, dtype=torch.float64),
                torch.tensor(d_table * gv, dtype=torch.float64), None)


def witness_gain(ctx: "B.Context", theta, table, z, gamma: float, witness: "B.Beam", dt: float,
                 ppc: int, r_max: float, checkpoint_every: int = 0, schedule=None):
    """L(theta, table) as a differentiable torch scalar (float64, CPU).  With
    `schedule` (n_xi sub-step counts) the forward step replays it instead of
    choosing sub-steps adaptively; the loss is then smooth in its inputs."""
    prob = _Problem(ctx, z, gamma, witness, dt, ppc, r_max, checkpoint_every, schedule)
    return WitnessGain.apply(theta, table, prob)
