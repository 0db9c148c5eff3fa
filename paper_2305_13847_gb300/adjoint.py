"""Gradients through many time steps: binomial checkpointing and torch.autograd.

The forward steps and the adjoint of each step run in the CUDA library
(dg_step, dg_adjoint_step, dg_cloud_functional); this module only schedules
them.  Reversing n steps while holding at most s stored states uses the
binomial checkpointing schedule of Griewank ("revolve"; Griewank and
Walther, ACM TOMS 26, 2000): with t sweeps and s snapshots at most
beta(s, t) = C(s + t, s) steps can be reversed, and the reversal of n steps
splits into a tail of up to beta(s - 1, t) steps (reversed with one snapshot
fewer) and a head of the remaining steps (one sweep fewer).
"""
import math

import torch

from . import dgmoist as dm


def beta(s, t):
    return math.comb(s + t, s)


class Stepper:
    """Forward steps and step adjoints of one context on device tensors."""

    def __init__(self, ctx, dt):
        self.ctx = ctx
        self.dt = float(dt)
        self.forward_steps = 0
        self.adjoint_steps = 0
        self.max_held = 0
        self._held = 0

    def advance(self, U, m):
        out = torch.empty_like(U)
        dm.dg_set_state(self.ctx, U, dm.DG_DEVICE)
        dm.dg_step(self.ctx, self.dt, int(m))
        dm.dg_get_state(self.ctx, out, dm.DG_DEVICE)
        self.forward_steps += int(m)
        return out

    def adjoint(self, U, lam):
        out = torch.empty_like(lam)
        dm.dg_adjoint_step(self.ctx, self.dt, U, lam, out)
        self.adjoint_steps += 1
        return out

    def hold(self, k):
        self._held += k
        self.max_held = max(self.max_held, self._held)


def revolve_adjoint(stepper, U0, n, snapshots, lam_n):
    """lam_0 = (dU_n / dU_0)^T lam_n with at most `snapshots` states held
    besides U0 (binomial schedule, module docstring)."""

    def rec(U_start, n, s, lam):
        if n == 0:
            return lam
        if n == 1:
            return stepper.adjoint(U_start, lam)
        if s == 0:
            for i in range(n - 1, -1, -1):
                Ui = stepper.advance(U_start, i) if i else U_start
                lam = stepper.adjoint(Ui, lam)
            return lam
        t = 1
        while beta(s, t) < n:
            t += 1
        m = max(1, n - beta(s - 1, t))
        U_mid = stepper.advance(U_start, m)
        stepper.hold(1)
        lam = rec(U_mid, n - m, s - 1, lam)
        del U_mid
        stepper.hold(-1)
        return rec(U_start, m, s, lam)

    return rec(U0, int(n), int(snapshots), lam_n)


class DGSteps(torch.autograd.Function):
    """U_n = (SSPRK(4,3) step)^n (U_0); backward by revolve + dg_adjoint_step."""

    @staticmethod
    def forward(fctx, U0, stepper, nsteps, snapshots):
        fctx.stepper = stepper
        fctx.nsteps = int(nsteps)
        fctx.snapshots = int(snapshots)
        fctx.save_for_backward(U0)
        return stepper.advance(U0.detach().contiguous(), nsteps)

    @staticmethod
    def backward(fctx, grad_out):
        (U0,) = fctx.saved_tensors
        lam0 = revolve_adjoint(fctx.stepper, U0.detach().contiguous(), fctx.nsteps,
                               fctx.snapshots, grad_out.contiguous())
        return lam0, None, None, None


class CloudWater(torch.autograd.Function):
    """J(U) = integral of the cloud density rho_c over the domain."""

    @staticmethod
    def forward(fctx, U, ctx):
        grad = torch.empty_like(U)
        J = dm.dg_cloud_functional(ctx, U.detach().contiguous(), grad)
        fctx.save_for_backward(grad)
        return torch.tensor(J, dtype=U.dtype, device=U.device)

    @staticmethod
    def backward(fctx, gJ):
        (grad,) = fctx.saved_tensors
        return gJ * grad, None


def cloud_water_gradient(ctx, U0, dt, nsteps, snapshots=32):
    """J(U_n) and dJ/dU_0 for U_n after nsteps steps from U0 (device, float64).

    Returns (J, grad, stepper); grad has the layout of U0.
    """
    stepper = Stepper(ctx, dt)
    U = U0.detach().clone().requires_grad_(True)
    J = CloudWater.apply(DGSteps.apply(U, stepper, nsteps, snapshots), ctx)
    J.backward()
    return float(J.item()), U.grad, stepper
