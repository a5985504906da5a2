"""Seismogram misfit as a torch.autograd.Function.

J(rho, lambda, mu) = sum over shots s of 1/2 dt sum_n sum_r |P_r v_s^{n+1/2} - d_{s,r}^n|^2, each
shot a run from rest with its own point source.  The forward pass computes the misfit and its
gradient together by the discrete adjoint of the time step, all shots in one call
(slt_adjoint_batched: fields with the shots innermost, untiled or on the schedule's tiles); a
schedule the batched adjoint does not take falls back to one slt_adjoint call per shot.
Backward returns the stored gradient scaled by the incoming gradient.  Material tensors are
per-cell float64 (any device); they are copied to the mesh before the run.
"""
import numpy as np
import torch

from . import (SltError, slt_adjoint, slt_adjoint_batched, slt_mesh_info, slt_mesh_set_material,
               slt_mesh_set_source, slt_receivers_create)


class MisfitProblem:
    """mesh, schedule (None = untiled), receiver positions [nrec, 2], shot positions [nshots, 2],
    observed data [nshots, nsteps, nrec, 2] (CUDA float64), source series [nsteps] (CUDA float64),
    dt, nsteps, checkpoint interval."""

    def __init__(self, mesh, sched, rec_xy, shots_xy, data, ricker, dt, nsteps, checkpoint_every=50):
        self.mesh, self.sched = mesh, sched
        self.rec = slt_receivers_create(mesh, rec_xy)
        self.shots = np.asarray(shots_xy, dtype=np.float64).reshape(-1, 2)
        self.data, self.ricker = data, ricker
        self.dt, self.nsteps, self.k = float(dt), int(nsteps), int(checkpoint_every)
        self.ncell = slt_mesh_info(mesh)["ncell"]

    def __call__(self, rho, lam, mu):
        return SeismogramMisfit.apply(rho, lam, mu, self)


class SeismogramMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, lam, mu, problem):
        host = [t.detach().to("cpu", torch.float64).numpy() for t in (rho, lam, mu)]
        slt_mesh_set_material(problem.mesh, *host)
        total = 0.0
        grad = torch.zeros((3, problem.ncell), dtype=torch.float64, device="cuda")
        batched = problem.k >= 1
        if batched:
            try:
                data = problem.data.permute(1, 0, 2, 3).contiguous()   # [nsteps, nshots, nrec, 2]
                total = slt_adjoint_batched(problem.mesh, problem.sched, problem.rec, problem.shots, problem.ricker,
                                            problem.dt, problem.nsteps, data, problem.k, grad)
            except SltError as e:
                if e.code != -6:   # a schedule the batched adjoint does not take
                    raise
                batched = False
        if not batched:
            g = torch.empty_like(grad)
            for s, xy in enumerate(problem.shots):
                slt_mesh_set_source(problem.mesh, xy)
                total += slt_adjoint(problem.mesh, problem.sched, problem.rec, problem.ricker, problem.dt,
                                     problem.nsteps, problem.data[s], problem.k, g)
                grad += g
        ctx.save_for_backward(grad)
        ctx.devices = [t.device for t in (rho, lam, mu)]
        return torch.tensor(total, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        out = [(gJ.to(grad.device) * grad[k]).to(ctx.devices[k]) for k in range(3)]
        return out[0], out[1], out[2], None
