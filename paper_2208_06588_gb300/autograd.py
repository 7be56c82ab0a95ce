"""torch.autograd.Function over swale_adjoint (argument marshalling only).

gauge_misfit(eta0, hu0, b0, ...) returns the gauge misfit J (one value per instance) of
nsteps SSP-RK3 steps (Eq. RK32D) of the well-balanced ALE-WENO scheme from the initial cell
averages; J.backward() delivers dJ/d(eta0, hu0, b0) of the discrete scheme, computed by the
CUDA adjoint in the same call that evaluates J (dt and the stage viscosities of the forward
run are held fixed, as are the detector classes and limiter branches). The misfit is
    J_i = sum_n dt_n sum_g (h(gauge g of instance i, t_n) - h_obs[n][i][g])^2.
Inputs must be CUDA tensors; nothing here runs on the CPU.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def _f64(t, dev):
    if not torch.is_tensor(t):
        t = torch.as_tensor(np.asarray(t))
    return t.detach().to(device=dev, dtype=torch.float64).contiguous()


class GaugeMisfit(torch.autograd.Function):
    """Forward: J (B values) and the three gradients in one swale_adjoint call. Backward: the
    gradients scaled by the incoming dJ of the instance that owns each cell."""

    @staticmethod
    def forward(ctx, eta0, hu0, b0, x_nodes, profile, gauges_x, h_obs, cfg, nsteps, ckpt_every, offsets, cfl, tape):
        dev = eta0.device
        if dev.type != "cuda":
            raise ValueError("gauge_misfit runs on CUDA tensors only")
        E, M, Bt = (_f64(t, dev) for t in (eta0, hu0, b0))
        x = _f64(x_nodes, dev)
        prof = None if profile is None else _f64(profile, dev)
        gx, obs = _f64(gauges_x, dev), _f64(h_obs, dev)
        if offsets is None:
            nb, counts = 1, None
            off = None
        else:
            off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
            nb = off.size - 1
            counts = torch.as_tensor(np.diff(off), device=dev)
        G = gx.numel() // nb
        if G * nb != gx.numel() or obs.numel() != nsteps * nb * G:
            raise ValueError("gauges_x needs B*G values and h_obs nsteps*B*G values")
        J = torch.zeros(nb, dtype=torch.float64, device=dev)
        gE, gM, gB = torch.zeros_like(E), torch.zeros_like(E), torch.zeros_like(E)
        with torch.cuda.device(dev):
            solver = B.Solver(cfg, ctypes_stream(dev))
            try:
                if off is None:
                    B.swale_set_problem(solver.ctx, E.numel(), x, E, M, Bt, prof, 1)
                else:
                    c = None if cfl is None else np.ascontiguousarray(np.asarray(cfl, dtype=np.float64))
                    B.swale_batch_set_problem(solver.ctx, nb, off, x, E, M, Bt, prof, c, 1)
                B.swale_set_adjoint_tape(solver.ctx, 1 if tape else 0)
                B.swale_adjoint(solver.ctx, nsteps, ckpt_every, G, gx, obs, J, gE, gM, gB)
            finally:
                solver.close()
        ctx.save_for_backward(gE, gM, gB)
        ctx.counts = counts
        return J

    @staticmethod
    def backward(ctx, gJ):
        gE, gM, gB = ctx.saved_tensors
        w = gJ[0] if ctx.counts is None else torch.repeat_interleave(gJ, ctx.counts)
        return (w * gE, w * gM, w * gB) + (None,) * 10


def ctypes_stream(dev):
    """The raw handle of torch's current stream on ``dev`` (the solver works in its order)."""
    return torch.cuda.current_stream(dev).cuda_stream


def gauge_misfit(eta0, hu0, b0, x_nodes, profile, gauges_x, h_obs, cfg, nsteps, ckpt_every=64, offsets=None,
                 cfl=None, tape=False):
    """J[B] of nsteps steps from (eta0, hu0, b0); differentiable in the three initial fields.

    x_nodes / profile: N+1 nodes per instance (concatenated for a batch, as in
    swale_batch_set_problem); gauges_x: B*G positions; h_obs: nsteps x B x G observed depths;
    offsets: B+1 cell offsets of a batch (None: one instance); cfl: per-instance CFL numbers;
    tape: keep each step's stage data instead of recomputing it (swale_set_adjoint_tape)."""
    return GaugeMisfit.apply(eta0, hu0, b0, x_nodes, profile, gauges_x, h_obs, cfg, nsteps, ckpt_every, offsets,
                             cfl, tape)
