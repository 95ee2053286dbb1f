"""torch.autograd front end of the training path.

``enhanced_nms(llr, alpha, code, autos)`` runs the enhanced NMS iterations of
Algorithm 1 (no early stop, checkpoint of y^(t) after every iteration) with the
per-iteration normalization factors alpha_t of Eq. (3), and differentiates through
them with the library's backward kernel (subgradient of min-sum: d c2v / d alpha_t =
c2v / alpha_t, d c2v / d |z| only at the minimum).  ``bce(y, codeword)`` is the
binary cross-entropy of the final LLRs against the transmitted word, on the library's
loss kernel.  Both are thin wrappers: the arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import bchdec as B


class EnhancedNms(torch.autograd.Function):
    """y^(I) = NMS(llr; alpha_1..alpha_I) with checkpoints; gradients for llr and alpha."""

    @staticmethod
    def forward(ctx, llr, alpha, code, autos, n_autos):
        if llr.dtype != torch.float32 or not llr.is_cuda:
            raise ValueError("llr must be a float32 CUDA tensor [F][ld]")
        if autos.dtype != torch.int16 or not autos.is_cuda:
            raise ValueError("autos must be an int16 CUDA tensor [F][n_autos]")
        I = int(alpha.numel())
        p = B.params(I, alpha.detach().float().cpu().numpy(), n_autos=n_autos, early_stop=False)
        llr = llr.contiguous()
        F, ld = llr.shape
        ckpt = torch.empty((I + 1, F, ld), dtype=torch.float32, device=llr.device)
        ws = B.workspace(code, p, F, device=llr.device)
        B.nms_forward_train(code, p, llr, autos, ckpt, ws)
        ctx.save_for_backward(autos, ckpt)
        ctx.code, ctx.p, ctx.ws = code, p, ws
        ctx.alpha_device, ctx.alpha_dtype = alpha.device, alpha.dtype
        return ckpt[I].clone()

    @staticmethod
    def backward(ctx, grad_y):
        autos, ckpt = ctx.saved_tensors
        grad_y = grad_y.contiguous().float()
        F, ld = grad_y.shape
        gl = torch.empty((F, ld), dtype=torch.float32, device=grad_y.device) \
            if ctx.needs_input_grad[0] else None
        ga = torch.empty(ctx.p.iters, dtype=torch.float32, device=grad_y.device)
        B.nms_backward(ctx.code, ctx.p, autos, ckpt, grad_y, gl, ga, ctx.ws)
        ga = ga.to(device=ctx.alpha_device, dtype=ctx.alpha_dtype) if ctx.needs_input_grad[1] else None
        return gl, ga, None, None, None


class BceLoss(torch.autograd.Function):
    """mean_i softplus(-(1 - 2 c_i) y_i) over frames and the n code bits."""

    @staticmethod
    def forward(ctx, y, codeword, code):
        y = y.contiguous().float()
        F, ld = y.shape
        loss = torch.empty(1, dtype=torch.float32, device=y.device)
        grad = torch.empty((F, ld), dtype=torch.float32, device=y.device)
        ws = B.workspace(code, B.params(1, 1.0), F, device=y.device)
        B.bce_loss(code.n, y, codeword, loss, grad, ws)
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None, None


def enhanced_nms(llr, alpha, code, autos, n_autos=None):
    """Differentiable enhanced NMS; ``alpha`` is a tensor of the I per-iteration factors."""
    return EnhancedNms.apply(llr, alpha, code, autos, int(n_autos or autos.shape[1]))


def bce(y, codeword, code):
    """Differentiable BCE of final LLRs ``y`` [F][ld] against packed codewords [F][words]."""
    return BceLoss.apply(y, codeword, code)


def alpha_init(iters, value=0.78, device="cuda"):
    return torch.tensor(np.full(iters, value, np.float32), device=device, requires_grad=True)
