"""torch.autograd binding of the diffusion-form stencils.

``DiffusionFn.apply(u0, coeff, nsteps, name, bc, checkpoint_every)`` returns
u_T after ``nsteps`` sweeps of the builtin ``name`` ("jacobi5", "diff7",
"star9r2") with coefficient ``coeff`` (a 0-d tensor).  The forward pass stores
a checkpoint every ``checkpoint_every`` steps (lope_forward_ckpt); the backward
pass recomputes each segment from its checkpoint and runs the transposed
stencil backward in time (lope_vjp), returning dL/du0 and dL/dc with dL/dc
accumulated in FP64 on the device.
"""
from __future__ import annotations

import torch

from . import _lib as L

_DT = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16"}


class DiffusionFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, coeff, nsteps, name="diff7", bc=None, checkpoint_every=10):
        u0 = u0.contiguous()
        c = float(coeff.detach().reshape(()).item())
        grid = L.Grid(u0.shape, _DT[u0.dtype], halo=2 if name == "star9r2" else 1)
        if bc is not None:
            grid.set_boundaries(bc)
        st = L.Stencil.builtin(name, c)
        uT, ws = L.forward_ckpt(grid, st, u0, nsteps, checkpoint_every)
        ctx.save_for_backward(u0)
        ctx.grid, ctx.st, ctx.ws = grid, st, ws
        ctx.nsteps, ctx.ckpt, ctx.coeff_shape, ctx.coeff_dtype = (nsteps, checkpoint_every,
                                                                  coeff.shape, coeff.dtype)
        return uT

    @staticmethod
    def backward(ctx, grad_uT):
        (u0,) = ctx.saved_tensors
        g, gc = L.vjp(ctx.grid, ctx.st, u0, grad_uT.to(u0.dtype).contiguous(), ctx.nsteps,
                      ctx.ckpt, reuse=True, workspace=ctx.ws)
        return g, gc.to(ctx.coeff_dtype).reshape(ctx.coeff_shape), None, None, None, None
