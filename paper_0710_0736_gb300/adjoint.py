"""torch.autograd bridge for the adjoint of T time steps.

SegmentationSteps.apply(image, lam, eps, u0, tau, steps, every, tol, precision)
returns u^T (the phase field after `steps` time steps, computed on the GPU by
libac) and, in backward, the gradients with respect to the image, lambda,
eps (tau held fixed) and u0 computed by libac's adjoint (ac_adjoint_backward):
every step is differentiated with its active set frozen and its adjoint
system solved by the same truncated V-cycle, with the forward recomputed from
checkpoints every `every` steps.  Argument marshalling only.
"""
from __future__ import annotations

import torch

from . import ac


class SegmentationSteps(torch.autograd.Function):
    @staticmethod
    def forward(fctx, image, lam, eps, u0, tau, steps, every, tol=1e-12, precision=ac.AC_FP64):
        H, W, _ = image.shape
        N = u0.shape[1]
        seg = ac.Segmenter(W, H, N, float(eps), float(lam), float(tau), tol=tol, precision=precision,
                           max_cycles=2000)
        if precision == ac.AC_MIXED:
            seg.set_image(image.detach().to(torch.float32).contiguous())
        else:
            seg.set_image(image.detach().to(torch.float64).contiguous())
        seg.set_phase(u0.detach().to(torch.float64).contiguous())
        ac.ac_adjoint_forward(seg.ctx, steps, every)
        uT = torch.empty((seg.n_nodes, N), dtype=torch.float64, device=image.device)
        ac.ac_get_phase(seg.ctx, uT, seg.n_nodes, N)
        torch.cuda.synchronize()
        fctx.seg = seg
        fctx.image_dtype = image.dtype
        return uT

    @staticmethod
    def backward(fctx, grad_uT):
        seg = fctx.seg
        dev = grad_uT.device
        g_img = torch.empty((seg.H, seg.W, 3), dtype=torch.float64, device=dev)
        g_u0 = torch.empty((seg.n_nodes, seg.N), dtype=torch.float64, device=dev)
        gl, ge = ac.ac_adjoint_backward(seg.ctx, grad_uT.detach().to(torch.float64).contiguous(), g_img, g_u0)
        torch.cuda.synchronize()
        seg.close()
        return (g_img.to(fctx.image_dtype), torch.tensor(gl, dtype=torch.float64, device=dev),
                torch.tensor(ge, dtype=torch.float64, device=dev), g_u0, None, None, None, None, None)


def misfit_loss(uT, m0, target):
    """L = 1/2 sum_n Mhat_n |u^T_n - onehot(target_n)|^2 (torch, differentiable)."""
    onehot = torch.nn.functional.one_hot(target.reshape(-1).long(), uT.shape[1]).to(uT.dtype)
    d = uT - onehot
    return 0.5 * (m0[:, None] * d * d).sum()
