"""Differentiable stage (b): the warp as a torch.autograd.Function whose backward is the hand-written adjoint.

Forward splats and gathers in the CUDA kernels (exw_splat_motion + exw_warp).  Backward calls exw_warp_backward,
which returns dL/d colour and dL/d motion with every integer decision of the forward pass held fixed (target,
winner, taps, tap participation, mask).  With ``checkpoint=True`` the splat keys are not kept between the passes
(8 bytes per pixel); the backward recomputes them into its workspace.  Depth receives no gradient: it only enters
integer decisions.
"""
from __future__ import annotations

import torch

from . import binding


class ExWarpFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, color, depth, mv, k: int, denom: int, checkpoint: bool):
        keys = binding.exw_splat_motion(depth, mv, k, denom)
        out, mask = binding.exw_warp(color, depth, mv, keys, k, denom)
        if checkpoint:
            ctx.save_for_backward(color, depth, mv)
        else:
            ctx.save_for_backward(color, depth, mv, keys)
        ctx.k, ctx.denom, ctx.checkpoint = int(k), int(denom), bool(checkpoint)
        ctx.mark_non_differentiable(mask)
        return out, mask

    @staticmethod
    def backward(ctx, grad_out, grad_mask):
        saved = ctx.saved_tensors
        color, depth, mv = saved[:3]
        keys = None if ctx.checkpoint else saved[3]
        g = grad_out.to(torch.float32).contiguous()
        gc, gm = binding.exw_warp_backward(g, color, depth, mv, keys, ctx.k, ctx.denom)
        gcol = gc.to(color.dtype) if ctx.needs_input_grad[0] else None
        gmv = gm if ctx.needs_input_grad[2] else None
        return gcol, None, gmv, None, None, None


def warp(color, depth, mv, k: int, denom: int = 4, checkpoint: bool = True):
    """Differentiable warp of ``color`` [3][H][W] by fraction k/denom of ``mv`` [2][H][W]: (out, mask)."""
    return ExWarpFunction.apply(color, depth, mv, k, denom, checkpoint)
