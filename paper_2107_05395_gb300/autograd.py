"""torch.autograd.Function over the checkpointed rollout of the C ABI.

    C_T = SharedLHSRollout.apply(C0, p, kind, N, dt, nsteps, ckpt_every[, bc, group])

C0 is an (N, M) FP64 CUDA tensor of initial states (interleaved, system fastest),
p a 0-dim FP64 tensor with the stepper coefficient (r for diffusion /
hyperdiffusion, gamma in grid units for Cahn-Hilliard).  Backward returns
dL/dC0 and dL/dp from the library's adjoint kernels (A^T solves with the same
shared factors); the shared matrix depends on p, so each call factorises it for
the given value.  When the batch is sharded over ranks (``group`` a process group,
each rank holding its own systems and a loss normalised by the global batch),
dL/dp is summed over the ranks in rank order; dL/dC0 stays local.  Marshalling
only: every step runs in libsbsolve.
"""
from __future__ import annotations

import torch

from . import _lib
from .distributed import sum_in_rank_order

_SCHEME_FOR = {"diffusion": ("be", "dirichlet"), "hyperdiffusion": ("be", "hinged"),
               "cahn_hilliard": ("be", "noflux")}


class SharedLHSRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, C0, p, kind, N, dt, nsteps, ckpt_every, bc=None, group=None):
        if C0.dtype != torch.float64 or not C0.is_cuda or C0.dim() != 2 or C0.shape[0] != N:
            raise ValueError("C0 must be an (N, M) float64 CUDA tensor")
        scheme, default_bc = _SCHEME_FOR[kind]
        st = _lib.sb_stepper_create(kind, scheme, bc or default_bc, N, float(p.item()), dt)
        C0c = C0.contiguous()
        M = C0c.shape[1]
        work = torch.empty(_lib.sb_rollout_workspace_bytes(st, M, nsteps, ckpt_every) // 8,
                           dtype=torch.float64, device=C0.device)
        CT = torch.empty_like(C0c)
        _lib.sb_rollout_forward(st, C0c, CT, nsteps, ckpt_every, work)
        ctx.st, ctx.work, ctx.nsteps, ctx.k, ctx.group = st, work, nsteps, ckpt_every, group
        return CT

    @staticmethod
    def backward(ctx, grad_CT):
        g = grad_CT.contiguous().to(torch.float64)
        grad_C0 = torch.empty_like(g)
        grad_p = torch.zeros((), dtype=torch.float64, device=g.device)
        _lib.sb_rollout_backward(ctx.st, g, grad_C0, ctx.nsteps, ctx.k, ctx.work, grad_param=grad_p)
        if ctx.group is not None:
            grad_p = sum_in_rank_order(grad_p, ctx.group)
        ctx.st = ctx.work = None
        return grad_C0, grad_p, None, None, None, None, None, None, None
