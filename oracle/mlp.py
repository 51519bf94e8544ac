"""Stages (b) and (c): BRDF decoder B and implicit ray tracer I  (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Both are MLPs with "3 layers in total with hidden dimensions set to 64"
(Sec. 4.1): y = W3 ReLU(W2 ReLU(W1 z + b1) + b2) + b3 (reading: biases
present; they are zero in the synthetic scenes unless a test sets them).

B (Sec. 3.2 and Sec. 3.3): z = f; the output vector is [n, a, r]
(treated "as one concatenated output vector"), then n <- n / ||n||,
a <- sigmoid(a), r <- 0.09 + 0.91 sigmoid(r).

I (Sec. 3.2 and Sec. 3.3): z = [f, PE(w)] with PE(w) = [w, sin(2^k pi w),
cos(2^k pi w)] for k = 0..3 (27 values; reading: the raw direction is
included and the frequency count is 4); outputs v = sigmoid(z0) and
t_hat = softplus(z1); the depth is min-max normalised between near and far
and clamped to 1 (= far), so t = near + (far - near) * min(t_hat, 1).

Pins (tests/test_oracle_mlp.py): the MLP against a numpy float64 matmul
chain; sigmoid/softplus at known points; the positional encoding against
its closed-form values at w = 0 and at the axes; the depth mapping at its
end points.

Kernel arithmetic (`mlp3_arith`), used only where floating point decides an
integer: the hard-visibility hit test 1[z0 > 0] of the paper's inference is
taken on the logit as a kernel computes it.  'bf16' rounds the layer
inputs, the two hidden weight matrices and the first hidden activations to
bfloat16 (round to nearest even) and keeps the biases and the output layer
in float32, with float64 sums (the tensor cores' float32 accumulation
differs from them only in summation order); 'bf16x3' is the split form of
the BF16 kernels' primary evaluation of I: each of those bf16 operands is a
bf16 hi part plus a bf16 lo part (the rounding residual) and every product
a.w is taken as a_hi w_hi + a_lo w_hi + a_hi w_lo, dropping only a_lo w_lo;
'fp32' rounds every operand and every layer result to float32.  Pins: exact
agreement with `mlp3` when all roundings are exact, and the rounding of each
stage observed on values that are not representable (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import torch

Layers = Sequence[Tuple[torch.Tensor, torch.Tensor]]

N_FREQ = 4
PE_DIM = 3 + 2 * 3 * N_FREQ   # 27


def as_layers(layers) -> List[Tuple[torch.Tensor, torch.Tensor]]:
    """Convert (W, b) array pairs to float64 tensors."""
    return [(torch.as_tensor(w, dtype=torch.float64), torch.as_tensor(b, dtype=torch.float64))
            for w, b in layers]


def _jit(x: torch.Tensor, jitter) -> torch.Tensor:
    """Conditioning probe only: x (1 + rel z), z ~ N(0, 1) from generator g."""
    if jitter is None:
        return x
    rel, g = jitter
    return x * (1.0 + rel * torch.randn(x.shape, generator=g, dtype=x.dtype))


def mlp3(z: torch.Tensor, layers: Layers, jitter=None) -> torch.Tensor:
    """Three linear layers with ReLU after the first two.

    `jitter` = (rel, torch.Generator) perturbs the input and both hidden
    activations by relative Gaussian noise; it is used only by the
    conditioning probe ``render.float32_sensitivity``.
    """
    (w1, b1), (w2, b2), (w3, b3) = layers
    h1 = torch.relu(_jit(z, jitter) @ w1.T + b1)
    h2 = torch.relu(_jit(h1, jitter) @ w2.T + b2)
    return _jit(h2, jitter) @ w3.T + b3


def round_to(x: torch.Tensor, arith: str) -> torch.Tensor:
    """x rounded to a narrower IEEE format (round to nearest even), returned in float64."""
    dt = {"bf16": torch.bfloat16, "fp16": torch.float16, "fp32": torch.float32}[arith]
    return x.to(dt).to(torch.float64)


def mlp3_arith(z: torch.Tensor, layers: Layers, arith: str) -> torch.Tensor:
    """mlp3 in a kernel's arithmetic ('bf16', 'bf16x3' or 'fp32'; see the module notes)."""
    (w1, b1), (w2, b2), (w3, b3) = layers
    if arith == "bf16":
        r16 = lambda a: round_to(a, "bf16")
        r32 = lambda a: round_to(a, "fp32")
        h1 = r32(torch.relu(r16(z) @ r16(w1).T + r32(b1)))
        h2 = r32(torch.relu(r16(h1) @ r16(w2).T + r32(b2)))
        return r32(h2 @ r32(w3).T + r32(b3))
    if arith == "bf16x3":
        r16 = lambda a: round_to(a, "bf16")
        r32 = lambda a: round_to(a, "fp32")

        def mm(a, w):
            ah, wh = r16(a), r16(w)
            al, wl = r16(a - ah), r16(w - wh)
            return ah @ wh.T + al @ wh.T + ah @ wl.T
        h1 = r32(torch.relu(mm(z, w1) + r32(b1)))
        h2 = r32(torch.relu(mm(h1, w2) + r32(b2)))
        return r32(h2 @ r32(w3).T + r32(b3))
    if arith == "fp32":
        f = lambda a: a.to(torch.float32)
        h1 = torch.relu(f(z) @ f(w1).T + f(b1))
        h2 = torch.relu(h1 @ f(w2).T + f(b2))
        return (h2 @ f(w3).T + f(b3)).to(torch.float64)
    raise ValueError(arith)


def brdf_decoder(f: torch.Tensor, layers: Layers, jitter=None):
    """a, r, n = B(f): albedo [.,3], roughness [.], unit normal [.,3]."""
    y = mlp3(f, layers, jitter)
    n = y[:, 0:3]
    n = n / n.norm(dim=1, keepdim=True).clamp(min=1e-12)
    a = torch.sigmoid(y[:, 3:6])
    r = 0.09 + 0.91 * torch.sigmoid(y[:, 6])
    return a, r, n


def positional_encoding(w: torch.Tensor) -> torch.Tensor:
    """PE(w) = [w, sin(pi w), cos(pi w), sin(2 pi w), cos(2 pi w), ..., k = 0..3]."""
    parts = [w]
    for k in range(N_FREQ):
        arg = (2.0 ** k) * math.pi * w
        parts.append(torch.sin(arg))
        parts.append(torch.cos(arg))
    return torch.cat(parts, dim=-1)


def depth_from_logit(t_hat: torch.Tensor, near: float, far: float) -> torch.Tensor:
    """t = near + (far - near) * min(t_hat, 1): normalised depth clamped to far."""
    return near + (far - near) * torch.clamp(t_hat, max=1.0)


def implicit_ray_tracer(f: torch.Tensor, w: torch.Tensor, layers: Layers,
                        near: float, far: float, jitter=None):
    """v, t = I(f, w): soft visibility in (0, 1) and expected depth in [near, far]."""
    y = mlp3(torch.cat([f, positional_encoding(w)], dim=-1), layers, jitter)
    v = torch.sigmoid(y[:, 0])
    t = depth_from_logit(torch.nn.functional.softplus(y[:, 1]), near, far)
    return v, t
