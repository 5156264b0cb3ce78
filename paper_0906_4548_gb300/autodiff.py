"""Gradients through a PM run: torch.autograd.Function wrappers over the C ABI.

Every forward and backward computation runs in the library's kernels:
dgp_zeldovich / dgp_zeldovich_adjoint (initial conditions from a linear
field), pm_step / pm_step_adjoint (the kick-drift-kick step with the
nonlinear field solve and its adjoint), and dgp_deposit + power_spectrum /
dgp_power_spectrum_adjoint (the P(k) loss).  The run keeps one particle state
every K steps; the backward pass replays each K-step segment forward from its
checkpoint and applies the step transposes in reverse.

The context must not reorder particles (dgp_params.sort_every = 0), since the
cotangents refer to particles by their index, and must use the nonlinear
gravity mode.  r_c is a constant of the context: no gradient with respect to
it is formed here.
"""

import torch

from . import dgp


def _parts(x, p):
    return dgp.particles(x[0], x[1], x[2], p[0], p[1], p[2])


class ZeldovichIC(torch.autograd.Function):
    """delta_L (n^3 device field) -> (x, p), each (3, n^3), one particle per cell in lattice order."""

    @staticmethod
    def forward(fctx, delta_l, ctx, vel_factor):
        n = delta_l.shape[0]
        x = torch.empty((3, n ** 3), dtype=delta_l.dtype, device=delta_l.device)
        p = torch.empty_like(x)
        dgp.dgp_zeldovich(ctx, delta_l.contiguous(), vel_factor, _parts(x, p))
        fctx.ctx, fctx.vf, fctx.shape = ctx, vel_factor, delta_l.shape
        return x, p

    @staticmethod
    def backward(fctx, xbar, pbar):
        xb = xbar.contiguous().clone() if xbar is not None else None
        pb = pbar.contiguous().clone() if pbar is not None else None
        if xb is None:
            xb = torch.zeros_like(pb)
        if pb is None:
            pb = torch.zeros_like(xb)
        out = torch.empty(fctx.shape, dtype=xb.dtype, device=xb.device)
        dgp.dgp_zeldovich_adjoint(fctx.ctx, _parts(xb, pb), fctx.vf, out)
        return out, None, None


class PMRun(torch.autograd.Function):
    """(x0, p0) -> (x, p) after the steps of `schedule` (scale factors a_0 < a_1 < ...),
    with a checkpoint every `every` steps."""

    @staticmethod
    def forward(fctx, x0, p0, ctx, schedule, every):
        x, p = x0.detach().clone(), p0.detach().clone()
        parts = _parts(x, p)
        nsteps = len(schedule) - 1
        checkpoints = []
        for i in range(nsteps):
            if i % every == 0:
                checkpoints.append((i, x.clone(), p.clone()))
            dgp.pm_step(ctx, parts, schedule[i], schedule[i + 1] - schedule[i])
        fctx.ctx, fctx.schedule, fctx.checkpoints = ctx, list(schedule), checkpoints
        return x, p

    @staticmethod
    def backward(fctx, xbar, pbar):
        ctx, sched = fctx.ctx, fctx.schedule
        nsteps = len(sched) - 1
        xb = xbar.contiguous().clone() if xbar is not None else None
        pb = pbar.contiguous().clone() if pbar is not None else None
        if xb is None:
            xb = torch.zeros_like(pb)
        if pb is None:
            pb = torch.zeros_like(xb)
        cot = _parts(xb, pb)
        bounds = [c[0] for c in fctx.checkpoints] + [nsteps]
        for s in reversed(range(len(fctx.checkpoints))):
            i0, cx, cp = fctx.checkpoints[s]
            i1 = bounds[s + 1]
            # replay the segment, keeping the start state of every step
            starts = [(cx.clone(), cp.clone())]
            x, p = cx.clone(), cp.clone()
            parts = _parts(x, p)
            dgp.dgp_reset(ctx)
            for i in range(i0, i1 - 1):
                dgp.pm_step(ctx, parts, sched[i], sched[i + 1] - sched[i])
                starts.append((x.clone(), p.clone()))
            for i in reversed(range(i0, i1)):
                sx, sp = starts[i - i0]
                dgp.pm_step_adjoint(ctx, _parts(sx, sp), sched[i], sched[i + 1] - sched[i], cot)
        return xb, pb, None, None, None


class PkLoss(torch.autograd.Function):
    """L = sum_b w_b (P_b - T_b)^2 for the P(k) (power_spectrum, nbins shells) of the
    CIC density contrast of the particles at positions x (3, Np)."""

    @staticmethod
    def forward(fctx, x, ctx, n, target, weights):
        import numpy as np
        xc = x.detach().contiguous()
        parts = _parts(xc, xc)
        delta = torch.empty((n, n, n), dtype=x.dtype, device=x.device)
        dgp.dgp_deposit(ctx, parts, delta)
        t = np.asarray(target, dtype=np.float64)
        w = np.asarray(weights, dtype=np.float64)
        _, P, _ = dgp.power_spectrum(ctx, delta, t.size)
        fctx.ctx, fctx.x, fctx.dldp = ctx, xc, 2.0 * w * (P - t)
        return torch.tensor(float(np.sum(w * (P - t) ** 2)), dtype=torch.float64)

    @staticmethod
    def backward(fctx, lbar):
        xb = torch.zeros_like(fctx.x)
        dgp.dgp_power_spectrum_adjoint(fctx.ctx, _parts(fctx.x, fctx.x), fctx.dldp * float(lbar),
                                       _parts(xb, xb))
        return xb, None, None, None, None
