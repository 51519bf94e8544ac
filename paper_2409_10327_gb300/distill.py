"""Online per-head distillation of the hash renderer (Sec. 3.3; supplementary "Training Details").

    d = Distiller(student, teacher, table, brdf_w, irt_w, env)
    terms = d.step(pos, normal)          # [3]: BRDF L1, visibility BCE, depth L1

Each step draws K stratified whole-sphere directions per point
(rt_distill_dirs), takes the teacher's heads from its stage kernels (rt_encode,
rt_decode, rt_trace), accumulates the student's per-head loss gradient
(rt_distill_backward) and applies Adam (rt_adam_step; learning rate 2e-3,
weight decay 1e-6 on the MLPs), then rebinds the student's parameters.  This
module only orders those calls and owns the parameter and moment buffers.
"""
from __future__ import annotations

import torch

from . import binding
from .binding import Renderer


class Distiller:
    def __init__(self, student: Renderer, teacher: Renderer, table: torch.Tensor, brdf_w: torch.Tensor,
                 irt_w: torch.Tensor, env: torch.Tensor, K: int = 1024, lr: float = 2e-3,
                 weight_decay: float = 1e-6):
        self.student, self.teacher = student, teacher
        self.params = [t.detach().clone().float().contiguous() for t in (table, brdf_w, irt_w)]
        self.decay = [0.0, weight_decay, weight_decay]          # the MLPs only
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.m1 = [torch.zeros_like(p) for p in self.params]
        self.m2 = [torch.zeros_like(p) for p in self.params]
        self.env, self.K, self.lr, self.t = env, K, lr, 0
        self.loss = torch.zeros(3, device=table.device, dtype=torch.float32)
        self.student.set_params(*self.params, env)

    def step(self, pos: torch.Tensor, normal: torch.Tensor, ray_offset: int = 0) -> torch.Tensor:
        P = pos.shape[0]
        dirs = self.student.distill_dirs(P, self.K, ray_offset)
        feat = self.teacher.encode(pos)
        brdf_t = self.teacher.decode(feat)
        vis_t, depth_t = self.teacher.trace(feat, dirs)
        for g in self.grads:
            g.zero_()
        self.loss.zero_()
        self.student.distill_backward(pos, normal, dirs, brdf_t, vis_t, depth_t, self.loss, *self.grads)
        self.t += 1
        for p, g, a, b, wd in zip(self.params, self.grads, self.m1, self.m2, self.decay):
            binding.adam_step(p, g, a, b, self.t, lr=self.lr, weight_decay=wd)
        self.student.set_params(*self.params, self.env)
        return self.loss
