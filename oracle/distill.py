"""Per-head distillation of the hash renderer (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The hash renderer is trained online against a teacher (Sec. 3.3 "Training
Procedure"; supplementary "Training Details"): for a batch of primary points
x with normals n and, per point, K directions drawn by stratified sampling
on the whole sphere,

  * f = H(x); (n', a', r') = B(f) after n/|n|, sigmoid and 0.09 + 0.91 sigmoid,
    with an L1 loss against the teacher's (n', a', r');
  * (z0, z1) = I(f, w): sigmoid(z0) against the teacher's visibility
    binarised at 0.5 with binary cross-entropy, and the min-max normalised
    depth min(softplus(z1), 1) against the teacher's with an L1 loss;
  * directions that are not front-facing (w . n <= 0) are left out;
  * Adam, learning rate 2e-3, weight decay 1e-6 on the MLPs.

Readings: the loss is the sum of three means: the BRDF L1 over points and
the 7 output components, and BCE and depth L1 each averaged over a point's
front-facing directions, then over points (a point with none adds 0).  The
teacher is a model of the same architecture (synthetic workload: random
weights), and its binarised visibility is the hit test 1[z0 > 0] taken on
its logit as the kernel computes it (decision_arith, as for hard
visibility).  Stratified sampling: K = S^2 cells of the unit square, one
point per cell at cell (k // S, k % S) plus the uniforms of counter
ray_id * K + k (SplitMix64, sampling.py), mapped to the sphere with
z = 1 - 2 u1, azimuth 2 pi u2.  Weight decay is the L2 form of PyTorch's
Adam: g + wd * p, on the MLP parameters only.

Pins (tests/test_oracle_distill.py): one point per stratum; BCE and L1 at
closed-form points; identical student and teacher give the closed-form
loss sum_k softplus(-|z0|); finite differences of the loss; an Adam step
against its closed form.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np
import torch

from . import hashgrid, mlp, sampling
from .render import Params


def stratified_sphere(ray_ids, K: int, seed: int) -> torch.Tensor:
    """[R, K, 3] stratified directions on the whole sphere (K = S^2)."""
    S = int(round(math.sqrt(K)))
    if S * S != K:
        raise ValueError("K must be a perfect square")
    ids = np.asarray(ray_ids, np.uint64)
    ctr = ids[:, None] * np.uint64(K) + np.arange(K, dtype=np.uint64)[None, :]
    xi1, xi2 = sampling.uniforms(seed, ctr)
    k = torch.arange(K, dtype=torch.float64)
    u1 = (torch.div(k, S, rounding_mode="floor") + xi1) / S
    u2 = (torch.remainder(k, S) + xi2) / S
    return sampling.uniform_sphere(u1, u2)


def _heads(x, w, prm: Params, opt, arith: Optional[str] = None):
    """(n', a', r') [R, 7] of B at x and the I logits (z0, z1) [R, K] along w [R, K, 3]."""
    res = hashgrid.level_resolutions(opt.levels, opt.base_res, opt.max_res)
    dense = hashgrid.dense_levels(res, 1 << opt.log2_T, opt.dense_coarse)
    R, K = w.shape[0], w.shape[1]
    if arith is None:
        f = hashgrid.encode(x, prm.table, res, dense)
        a, r, n = mlp.brdf_decoder(f, prm.brdf)
        z = mlp.mlp3(torch.cat([f[:, None, :].expand(R, K, f.shape[1]).reshape(R * K, -1),
                                mlp.positional_encoding(w.reshape(-1, 3))], -1), prm.irt)
        return torch.cat([n, a, r[:, None]], -1), z[:, 0].reshape(R, K), z[:, 1].reshape(R, K)
    tab = mlp.round_to(prm.table, "fp32")
    f = mlp.round_to(hashgrid.encode(x, tab, res, dense, fp32_grid=True), "fp32")
    z = mlp.mlp3_arith(torch.cat([f[:, None, :].expand(R, K, f.shape[1]).reshape(R * K, -1),
                                  mlp.positional_encoding(w.reshape(-1, 3))], -1), prm.irt, arith)
    return None, z[:, 0].reshape(R, K), None


def teacher_targets(x, n, w, teacher: Params, opt, decision_arith: str = "fp32"):
    """(brdf [R, 7], v [R, K] in {0, 1}, normalised depth [R, K]) of the teacher."""
    brdf, z0, z1 = _heads(x, w, teacher, opt)
    _, z0k, _ = _heads(x, w, teacher, opt, decision_arith)
    v = (z0k > 0).to(torch.float64)
    return brdf, v, torch.clamp(torch.nn.functional.softplus(z1), max=1.0)


def bce_with_logits(z: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """-[y log sigmoid(z) + (1 - y) log(1 - sigmoid(z))] in the form that cannot overflow."""
    return torch.clamp(z, min=0.0) - z * y + torch.log1p(torch.exp(-z.abs()))


def distill_loss(x, n, w, student: Params, targets, opt):
    """(total, (brdf L1, BCE, depth L1)) for points x [R, 3], normals n [R, 3], directions w [R, K, 3]."""
    brdf_t, v_t, d_t = targets
    brdf, z0, z1 = _heads(x, w, student, opt)
    front = ((w * n[:, None, :]).sum(-1) > 0).to(torch.float64)
    cnt = front.sum(-1)
    per = torch.where(cnt > 0, 1.0 / torch.clamp(cnt, min=1.0), torch.zeros_like(cnt))[:, None] * front
    R = x.shape[0]
    l_brdf = (brdf - brdf_t).abs().sum() / (7.0 * R)
    l_bce = (bce_with_logits(z0, v_t) * per).sum() / R
    l_depth = ((torch.clamp(torch.nn.functional.softplus(z1), max=1.0) - d_t).abs() * per).sum() / R
    return l_brdf + l_bce + l_depth, (l_brdf, l_bce, l_depth)


def distill_gradient(x, n, w, student: Params, targets, opt):
    """(loss terms as floats, g_table, g_brdf, g_irt) by float64 autograd."""
    tab = student.table.detach().clone().requires_grad_(True)
    brdf = [(a.detach().clone().requires_grad_(True), b.detach().clone().requires_grad_(True)) for a, b in student.brdf]
    irt = [(a.detach().clone().requires_grad_(True), b.detach().clone().requires_grad_(True)) for a, b in student.irt]
    p = Params(tab, brdf, irt, student.env)
    total, terms = distill_loss(x, n, w, p, targets, opt)
    total.backward()
    flat = lambda layers: torch.cat([torch.cat([a.grad.reshape(-1), b.grad.reshape(-1)]) for a, b in layers])
    return [float(t.detach()) for t in terms], tab.grad, flat(brdf), flat(irt)


def adam_step(p, g, m, v, step: int, lr=2e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """One Adam update with L2 weight decay folded into the gradient; returns (p, m, v)."""
    g = g + weight_decay * p
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
