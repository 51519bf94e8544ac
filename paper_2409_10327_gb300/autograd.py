"""torch.autograd.Function around rt_render_frame / rt_backward (argument marshalling only).

    out = render(renderer, gb, table, brdf_w, irt_w, env, pixel_offset=0)   # [P, 3]

The forward binds the parameters (rt_set_params) and runs the fused kernel;
the backward calls the hand-written adjoint kernel, which recomputes the
activations and accumulates gradients for the hash table and both packed MLP
blobs.  Sampled directions are constants of the estimator.
"""
from __future__ import annotations

from typing import Dict

import torch

from .binding import Renderer


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, table, brdf_w, irt_w, env, renderer: Renderer, gb: Dict[str, torch.Tensor],
                pixel_offset: int):
        renderer.set_params(table, brdf_w, irt_w, env)
        out = renderer.render_frame(gb, pixel_offset)
        ctx.renderer, ctx.gb, ctx.offset = renderer, gb, pixel_offset
        ctx.shapes = (table, brdf_w, irt_w)
        return out[:, :3]

    @staticmethod
    def backward(ctx, grad):
        table, brdf_w, irt_w = ctx.shapes
        g4 = torch.zeros(grad.shape[0], 4, device=grad.device, dtype=torch.float32)
        g4[:, :3] = grad
        g_table = torch.zeros(table.shape, device=table.device, dtype=torch.float32)
        g_brdf = torch.zeros_like(brdf_w, dtype=torch.float32)
        g_irt = torch.zeros_like(irt_w, dtype=torch.float32)
        ctx.renderer.backward(ctx.gb, g4, g_table, g_brdf, g_irt, ctx.offset)
        return g_table.to(table.dtype), g_brdf, g_irt, None, None, None, None


def render(renderer: Renderer, gb: Dict[str, torch.Tensor], table: torch.Tensor, brdf_w: torch.Tensor,
           irt_w: torch.Tensor, env: torch.Tensor, pixel_offset: int = 0) -> torch.Tensor:
    """Differentiable radiance [P, 3] of the G-buffer gb."""
    return _RenderFn.apply(table, brdf_w, irt_w, env, renderer, gb, pixel_offset)
