"""torch.autograd.Function around the C-ABI distance and its adjoint.

WeakDistance.apply(ctx, rule, verts, tris, s, precision, nu) returns the
squared H^{-s} distance D of the mesh (verts: (V, 3) float64 CUDA tensor,
tris: (T, 3) int32 CUDA tensor) to the reference measure nu. The forward call
runs wd_distance_grad_dev, which evaluates D and dD/dverts in the library's
kernels; backward scales the stored gradient by the incoming gradient.
"""
from __future__ import annotations

import torch

from . import WD_FP64, wd_distance_grad_dev


class WeakDistance(torch.autograd.Function):
    @staticmethod
    def forward(fctx, wctx, rule, verts, tris, s=1.0, precision=WD_FP64, nu=None):
        if verts.dtype != torch.float64 or not verts.is_cuda:
            raise TypeError("verts must be a float64 CUDA tensor")
        v = verts.detach().contiguous()
        t = tris.to(torch.int32).contiguous()
        out = torch.zeros(1, dtype=torch.float64, device=v.device)
        grad = torch.empty_like(v)
        handle = wctx.handle if hasattr(wctx, "handle") else wctx
        wd_distance_grad_dev(handle, rule, v, t, nu, s, precision, out, grad)
        fctx.save_for_backward(grad)
        return out[0]

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return None, None, g * grad, None, None, None, None


def weak_distance(wctx, rule, verts, tris, s=1.0, precision=WD_FP64, nu=None):
    return WeakDistance.apply(wctx, rule, verts, tris, s, precision, nu)
