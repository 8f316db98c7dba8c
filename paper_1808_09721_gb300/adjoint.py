"""Gradients through SSP2(222) or SSP3(332) IMEX runs as a torch.autograd.Function.

`ImexSteps.apply(prims0, sigma, workload, nsteps, ckpt_every, scheme)` advances the
workload's model from the primitives `prims0` ([n_prim][ny][nx] or [n_prim][nz][ny][nx]
float64 CUDA tensor; n_prim = 11 for one fluid, 16 for two fluids) with conductivity
`sigma` (0-d float64 tensor) and returns the final conserved state ([14] or [18] planes).
Its backward runs the library's discrete
adjoint (rmhd_record / rmhd_adjoint_step): checkpoints every `ckpt_every`
steps, recomputation per segment, implicit-function-theorem adjoints of the
per-cell implicit solves. Any functional written with torch ops on the
returned state can then be differentiated w.r.t. prims0 and sigma.
"""
from __future__ import annotations

import dataclasses

import torch

from .sim import Sim


class ImexSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, prims0, sigma, workload, nsteps: int, ckpt_every: int = 10, scheme: int = 0):
        wl = dataclasses.replace(workload, sigma=float(sigma))
        sim = Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y, wl.cfl,
                  wl.mu_e, wl.mu_p, wl.kappa, device=prims0.device, scheme=scheme, nz=wl.nz, zlim=wl.zlim,
                  bc_z=wl.bc_z)
        sim.set_prims(prims0.detach().contiguous())
        sim.record(nsteps, ckpt_every)
        sim.step(wl.dt, nsteps)
        sim.check()
        out = torch.empty((sim.nc,) + sim.shape, dtype=torch.float64, device=prims0.device)
        sim.cons(out=out)
        ctx.sim = sim
        return out

    @staticmethod
    def backward(ctx, grad_out):
        sim = ctx.sim
        gp = torch.empty((sim.np,) + sim.shape, dtype=torch.float64, device=grad_out.device)
        _, gs = sim.adjoint(grad_out.contiguous(), out=gp)
        return gp, torch.tensor(gs, dtype=torch.float64, device=grad_out.device), None, None, None, None
