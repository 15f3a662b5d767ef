"""torch.autograd.Function over the rasterizer.

The forward saves nothing per pixel beyond what the library keeps in its context (final
transmittance and last-contributor index per pixel); the backward re-traverses each pixel's
list back to front and rebuilds the transmittance from those two numbers, instead of the
paper's per-pixel replay cache S = {id, C_in, alpha} (Eq. 9, Sec. III-C).  If another render
ran on the same context in between, the backward first re-renders this forward's inputs
(recomputation), so interleaved forwards stay correct.
"""
from __future__ import annotations

import torch

from . import rasterizer as R


class RasterizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast: R.Rasterizer, cam, sh_degree: int, means, log_scales, quats,
                opacity_logits, sh):
        ts = [t.detach().contiguous() for t in (means, log_scales, quats, opacity_logits, sh)]
        n = ts[0].shape[1]
        g = R.tensors_struct(n, sh_degree, *ts)
        image = rast.render_struct(g, cam)
        ctx.rast, ctx.cam, ctx.sh_degree = rast, cam, sh_degree
        ctx.render_id = rast.render_id
        ctx.save_for_backward(*ts)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        rast = ctx.rast
        ts = ctx.saved_tensors
        n = ts[0].shape[1]
        g = R.tensors_struct(n, ctx.sh_degree, *ts)
        if rast.render_id != ctx.render_id:
            rast.render_struct(g, ctx.cam)
        grads = [torch.zeros_like(t) for t in ts]
        rast.backward_struct(grad_image.contiguous().float(),
                             R.tensors_struct(n, ctx.sh_degree, *grads))
        return (None, None, None, *grads)


def rasterize(rast: R.Rasterizer, cam, means, log_scales, quats, opacity_logits, sh,
              sh_degree: int | None = None) -> torch.Tensor:
    """Differentiable render of planar parameters ([3][n], [3][n], [4][n], [n], [3][K][n])."""
    if sh_degree is None:
        K = sh.shape[1]
        sh_degree = int(round(K ** 0.5)) - 1
    return RasterizeFn.apply(rast, cam, sh_degree, means, log_scales, quats, opacity_logits, sh)
