"""torch.autograd.Function over the library's checkpointed discrete adjoint.

    J = mean_hot_wall_nusselt(theta, ra, (nx, ny, nz), nsteps, ckpt=50)
    J.backward()          # theta.grad, ra.grad from the hand-written adjoint

J(theta, Ra) is the hot-wall Nusselt number averaged over steps 1..nsteps of
a cavity started from its initial condition (T linear in x plus the seeded
noise, fluid at rest) with hot-wall temperature field theta (ny*nz values,
j fastest, or an array [nz, ny]) and Rayleigh number Ra.  The forward pass
runs the steps on the GPU keeping a checkpoint every ckpt steps; the
backward pass recomputes each segment from its checkpoint and sweeps the
discrete adjoint of the step (cavity_adjoint_forward / _backward in the C
ABI).  The sweep runs in the forward form's arithmetic (FP64 after an FP64
forward; FP32 adjoint arrays with FP64 sums over nodes after an FP32-mixed
one); the gradients it returns are FP64 tensors either way.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (CAVITY_FP64, Cavity, cavity_adjoint_backward, cavity_adjoint_forward,
               cavity_set_wall_temperature)


class MeanHotWallNusselt(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, ra, shape, nsteps, ckpt, opts):
        nx, ny, nz = shape
        c = Cavity(nx, ny, nz, precision=opts["precision"], seed=opts["seed"], noise_amp=opts["noise"],
                   device=opts["device"], Ra=float(ra), Pr=opts["Pr"])
        wall = theta.detach().to("cpu", torch.float64).numpy().reshape(-1)
        cavity_set_wall_temperature(c.h, 0, np.ascontiguousarray(wall))
        J = cavity_adjoint_forward(c.h, int(nsteps), int(ckpt))
        ctx.cavity = c
        ctx.dims = (ny, nz)
        ctx.theta_meta = (theta.shape, theta.dtype, theta.device)
        ctx.ra_meta = (ra.dtype, ra.device) if torch.is_tensor(ra) else None
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        ny, nz = ctx.dims
        g, gra = cavity_adjoint_backward(ctx.cavity.h, ny, nz)
        ctx.cavity.close()
        scale = float(gJ)
        shape, dtype, device = ctx.theta_meta
        gtheta = torch.from_numpy(g * scale).reshape(shape).to(device=device, dtype=dtype)
        gra_t = None
        if ctx.ra_meta is not None:
            gra_t = torch.tensor(gra * scale, dtype=ctx.ra_meta[0], device=ctx.ra_meta[1])
        return gtheta, gra_t, None, None, None, None


def mean_hot_wall_nusselt(theta: torch.Tensor, ra, shape, nsteps: int, ckpt: int = 50,
                          precision: int = CAVITY_FP64, seed: int = 0, noise: float = 0.0, Pr: float = 0.71,
                          device: int = 0) -> torch.Tensor:
    opts = dict(precision=precision, seed=seed, noise=noise, Pr=Pr, device=device)
    return MeanHotWallNusselt.apply(theta, ra, tuple(shape), nsteps, ckpt, opts)
