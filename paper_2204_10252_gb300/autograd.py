"""torch.autograd.Function around the unrolled preconditioned FISTA solve.

forward:  y = pFISTA_unrolled(b; lambda, c) on every slice of a pp_batch
          (raw b, fixed L_s, `iters` iterations, checkpoints every
          `checkpoint_every` iterations), all in libpp's kernels.
backward: libpp's reverse pass (soft-threshold Jacobian in the Haar domain,
          Horner adjoint through the self-adjoint normal operator) gives the
          gradients with respect to b, lambda and the polynomial coefficients.
Complex gradients follow PyTorch's convention for real losses:
dLoss/dRe + i dLoss/dIm.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class UnrolledPFISTA(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, lam, coeffs, batch, iters, checkpoint_every):
        c = np.ascontiguousarray(coeffs.detach().to(torch.float64).cpu().numpy())
        d = len(c) - 1
        bc = b.contiguous()
        out = torch.empty(int(batch.image_off[-1]), dtype=torch.complex64, device=b.device)
        lam_f = float(lam)
        B.pp_batch_unrolled_forward(batch, bc, lam_f, iters, c, d, checkpoint_every, out)
        ctx.batch, ctx.iters, ctx.ce, ctx.c, ctx.lam = batch, iters, checkpoint_every, c, lam_f
        ctx.lam_meta = (lam.dtype, lam.device) if isinstance(lam, torch.Tensor) else None
        ctx.c_meta = (coeffs.dtype, coeffs.device)
        ctx.save_for_backward(bc)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (bc,) = ctx.saved_tensors
        gb = torch.empty_like(bc)
        gl, gc = B.pp_batch_unrolled_backward(ctx.batch, bc, ctx.lam, ctx.iters, ctx.c,
                                              len(ctx.c) - 1, ctx.ce, grad_out.contiguous(), gb)
        g_lam = None
        if ctx.lam_meta is not None:
            g_lam = torch.tensor(gl, dtype=ctx.lam_meta[0], device=ctx.lam_meta[1])
        g_c = torch.tensor(gc, dtype=ctx.c_meta[0], device=ctx.c_meta[1])
        return gb, g_lam, g_c, None, None, None


def unrolled_pfista(batch, b, lam, coeffs, iters: int, checkpoint_every: int = 5):
    """Differentiable unrolled solve; lam a scalar tensor, coeffs a [d+1]
    tensor (float64 recommended); returns the concatenated images."""
    return UnrolledPFISTA.apply(b, lam, coeffs, batch, iters, checkpoint_every)
