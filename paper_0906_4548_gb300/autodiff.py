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
gravity mode.

The crossover scale r_c H0 is a constant of the context; its gradient is
formed by passing it as a 0-dim float64 tensor equal to the context's value:
VelocityFactor (the Zel'dovich velocity factor a^2 E f, dgp_velocity_factor),
ZeldovichIC with that tensor as vel_factor (dgp_zeldovich_vf_adjoint), and
PMRun's `rc` argument (pm_step_adjoint_rc summed over the steps).
"""

import torch

from . import dgp


def _parts(x, p):
    return dgp.particles(x[0], x[1], x[2], p[0], p[1], p[2])


class VelocityFactor(torch.autograd.Function):
    """r_c H0 (0-dim float64 tensor) -> vf = a^2 E f at scale factor a (host, float64)."""

    @staticmethod
    def forward(fctx, rc, omega_m0, a):
        vf, dvf = dgp.dgp_velocity_factor(omega_m0, float(rc), a)
        fctx.dvf = dvf
        return torch.tensor(vf, dtype=torch.float64)

    @staticmethod
    def backward(fctx, vbar):
        return vbar * fctx.dvf, None, None


class ZeldovichIC(torch.autograd.Function):
    """delta_L (n^3 device field) -> (x, p), each (3, n^3), one particle per cell in lattice order."""

    @staticmethod
    def forward(fctx, delta_l, ctx, vel_factor):
        n = delta_l.shape[0]
        x = torch.empty((3, n ** 3), dtype=delta_l.dtype, device=delta_l.device)
        p = torch.empty_like(x)
        vf = float(vel_factor)
        dl = delta_l.detach().contiguous()
        dgp.dgp_zeldovich(ctx, dl, vf, _parts(x, p))
        fctx.ctx, fctx.vf, fctx.shape = ctx, vf, delta_l.shape
        fctx.vf_tensor = torch.is_tensor(vel_factor)
        fctx.dl = dl if fctx.vf_tensor else None
        return x, p

    @staticmethod
    def backward(fctx, xbar, pbar):
        xb = xbar.contiguous().clone() if xbar is not None else None
        pb = pbar.contiguous().clone() if pbar is not None else None
        if xb is None:
            xb = torch.zeros_like(pb)
        if pb is None:
            pb = torch.zeros_like(xb)
        vbar = None
        if fctx.vf_tensor:
            vbar = torch.tensor(dgp.dgp_zeldovich_vf_adjoint(fctx.ctx, fctx.dl, _parts(xb, pb)), dtype=torch.float64)
        out = torch.empty(fctx.shape, dtype=xb.dtype, device=xb.device)
        dgp.dgp_zeldovich_adjoint(fctx.ctx, _parts(xb, pb), fctx.vf, out)
        return out, None, vbar


class PMRun(torch.autograd.Function):
    """(x0, p0) -> (x, p) after the steps of `schedule` (scale factors a_0 < a_1 < ...),
    with a checkpoint every `every` steps.  rc: None, or the context's r_c H0 as a 0-dim
    float64 tensor whose gradient is wanted."""

    @staticmethod
    def forward(fctx, x0, p0, ctx, schedule, every, rc=None):
        x, p = x0.detach().clone(), p0.detach().clone()
        parts = _parts(x, p)
        nsteps = len(schedule) - 1
        checkpoints = []
        for i in range(nsteps):
            if i % every == 0:
                checkpoints.append((i, x.clone(), p.clone()))
            dgp.pm_step(ctx, parts, schedule[i], schedule[i + 1] - schedule[i])
        fctx.ctx, fctx.schedule, fctx.checkpoints = ctx, list(schedule), checkpoints
        fctx.want_rc = rc is not None
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
        rcbar = 0.0
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
                if fctx.want_rc:
                    rcbar += dgp.pm_step_adjoint_rc(ctx, _parts(sx, sp), sched[i], sched[i + 1] - sched[i], cot)
                else:
                    dgp.pm_step_adjoint(ctx, _parts(sx, sp), sched[i], sched[i + 1] - sched[i], cot)
        rc_grad = torch.tensor(rcbar, dtype=torch.float64) if fctx.want_rc else None
        return xb, pb, None, None, None, rc_grad


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
