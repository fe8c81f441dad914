"""torch.autograd.Function over the FAM time stepper (forward and adjoint kernels).

``evolve(U0, solver, nsteps, cfl, ckpt_every)`` advances the state U0 (a CUDA
float64 tensor in the library's layout) by nsteps FAM steps on the GPU and
returns U_T; its backward pass calls the library's adjoint (fam_adjoint:
checkpoints every ``ckpt_every`` steps, one recomputation per segment, step
sizes of the forward run held fixed) to return dJ/dU0 from dJ/dU_T.
The arithmetic of both directions runs in the CUDA kernels of libfam.so.
"""
from __future__ import annotations

import torch

from .fam import Solver


class FamEvolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0: torch.Tensor, solver: Solver, nsteps: int, cfl: float, ckpt_every: int):
        U0c = U0.detach().contiguous()
        solver.set_state(U0c)
        solver.run_steps(int(nsteps), float(cfl))
        UT = torch.empty_like(U0c)
        solver.get_state(UT)
        solver.sync()
        ctx.solver, ctx.nsteps, ctx.cfl, ctx.ckpt = solver, int(nsteps), float(cfl), int(ckpt_every)
        ctx.save_for_backward(U0c)
        return UT

    @staticmethod
    def backward(ctx, gUT: torch.Tensor):
        (U0,) = ctx.saved_tensors
        g = ctx.solver.adjoint(U0, gUT.contiguous(), ctx.nsteps, ctx.cfl, ctx.ckpt)
        torch.cuda.synchronize()
        return g, None, None, None, None


def evolve(U0: torch.Tensor, solver: Solver, nsteps: int, cfl: float, ckpt_every: int = 20) -> torch.Tensor:
    return FamEvolve.apply(U0, solver, nsteps, cfl, ckpt_every)
