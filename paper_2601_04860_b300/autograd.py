"""Differentiable fusion: a ``torch.autograd.Function`` over the CUDA kernels.

Forward folds the views into a ``VoxelFusion`` context and returns the fused
probability P (dense g^3 grid, or n_active for a sparse set).  Backward runs
the hand-written adjoint kernel (``divas_fuse_backward``), which recomputes
every vote per view -- nothing is stored between the passes except the
context's W and Z -- and scatters, with the gates held fixed,

    dL/dl   = dL/dP * (w / Z) * m (1 - m)            (mask logits)
    dL/dm   = dL/dP * (w / Z)                        (probability masks)
    dL/dD   = dL/dP * ((m - P) / Z) * w * 2 alpha1 e / Delta^2

into the pixel each vote read (derived from Eq. gs-depthweight and Eq.
compact-fusion).  The gates (in frame, mask >= tau, |e| <= Delta) are
piecewise constant: their derivative is zero almost everywhere.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .fusion import VoxelFusion


class DivasFuseFunction(torch.autograd.Function):
    """score = DivasFuseFunction.apply(fusion, cams, mask_type, n_views, *masks, *depths)."""

    @staticmethod
    def forward(ctx, fusion: VoxelFusion, cams, mask_type: int, n_views: int, *leaves):
        masks = [t.detach().contiguous() for t in leaves[:n_views]]
        depths = [t.detach().contiguous() for t in leaves[n_views:]]
        fusion.reset()
        fusion.add_views(cams, depths, masks, mask_type=mask_type)
        score = fusion.finalize(score=True)["score"]
        ctx.fusion = fusion
        ctx.stream = torch.cuda.current_stream()  # the backward runs on the forward's stream
        ctx.cams = cams
        ctx.mask_type = mask_type
        ctx.n_views = n_views
        ctx.save_for_backward(*masks, *depths)
        return score

    @staticmethod
    def backward(ctx, grad_score):
        saved = ctx.saved_tensors
        n = ctx.n_views
        masks, depths = list(saved[:n]), list(saved[n:])
        fusion: VoxelFusion = ctx.fusion
        if fusion.n_views != n:
            raise RuntimeError("the fusion context was modified between forward and backward")
        need_m = ctx.needs_input_grad[4:4 + n]
        need_d = ctx.needs_input_grad[4 + n:4 + 2 * n]
        st = ctx.stream  # grad_score was produced there by the loss's backward
        with torch.cuda.stream(st):
            gm = [torch.zeros_like(m) if need_m[k] else None for k, m in enumerate(masks)]
            gd = [torch.zeros_like(d) if need_d[k] else None for k, d in enumerate(depths)]
            g = grad_score.contiguous()
            for s0 in range(0, n, L.MAX_VIEWS_PER_CALL):
                s1 = min(n, s0 + L.MAX_VIEWS_PER_CALL)
                fusion.backward(ctx.cams[s0:s1], depths[s0:s1], masks[s0:s1], g,
                                grad_mask=gm[s0:s1], grad_depth=gd[s0:s1],
                                mask_type=ctx.mask_type, stream=st)
        return (None, None, None, None, *gm, *gd)


def fuse(fusion: VoxelFusion, cams, masks, depths, mask_type: int = L.MASK_LOGIT_F32):
    """Differentiable fused score P for views (masks[i], depths[i]) seen by cams[i].

    Gradients flow to every mask or depth tensor that requires grad.  The
    context must not fold other views between this call and ``backward``."""
    if len(cams) != len(masks) or len(cams) != len(depths):
        raise ValueError("cams, masks and depths must have the same length")
    return DivasFuseFunction.apply(fusion, list(cams), int(mask_type), len(cams), *masks,
                                   *depths)
