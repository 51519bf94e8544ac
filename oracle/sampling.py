"""Direction sampling  (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper samples the incoming light direction at the primary point (Eq. 1,
p(w_i) the pdf of the chosen sampler) and casts 8 random rays from each
secondary point (supplementary, "Rendering Details").  Readings:

  * both levels draw cosine-weighted directions about the local normal, so
    that (w . n) / p(w) = pi in Eq. 1 (the tiny-frame workload names
    cosine-weighted directions);
  * a cosine-weighted direction is built as w = normalize(n + s), s uniform
    on the unit sphere (the sphere |p - n| = 1 seen from the origin has
    solid-angle density proportional to cos(theta));  this map is
    continuous in n, unlike a tangent-frame construction;
  * the random numbers come from a counter-based generator: the k-th output
    (k >= 1) of SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) started at
    state = seed is mix(seed + k * 0x9E3779B97F4A7C15); a uniform is the top
    24 bits times 2^-24, exact in float32 and float64.

Counters: secondary sample id q = (pixel_offset + p) * N + i for the
primary direction i of pixel p; the primary direction uses slot 0, the j-th
direction at the secondary point x'_q uses slot 1 + j; slot c of sample q
has counter (q * (M + 1) + c) and draws outputs 2*counter + 1 and
2*counter + 2 for (u1, u2).

Pins (tests/test_oracle_sampling.py): the published SplitMix64 outputs for
seed 0; unit length and w . n >= 0; the cosine-lobe moments E[w.n] = 2/3,
E[(w.n)^2] = 1/2 and the uniform azimuth; uniformity of s on the sphere.
"""
from __future__ import annotations

import math

import numpy as np
import torch

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, k) -> np.ndarray:
    """The k-th output (k >= 1, array) of SplitMix64 started at state = seed."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform24(bits: np.ndarray) -> np.ndarray:
    """Top 24 bits of a 64-bit output scaled into [0, 1)."""
    return (bits >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


def counters(sample_id, slot, m_dirs: int) -> np.ndarray:
    """Counter of slot `slot` (0 = primary direction, 1 + j = secondary j) of sample q."""
    q = np.asarray(sample_id, dtype=np.uint64)
    return q * np.uint64(m_dirs + 1) + np.asarray(slot, dtype=np.uint64)


def uniforms(seed: int, ctr: np.ndarray):
    """(u1, u2) for counters ctr, as float64 tensors."""
    two = np.uint64(2)
    u1 = uniform24(splitmix64(seed, ctr * two + np.uint64(1)))
    u2 = uniform24(splitmix64(seed, ctr * two + np.uint64(2)))
    return torch.from_numpy(u1), torch.from_numpy(u2)


def uniform_sphere(u1: torch.Tensor, u2: torch.Tensor) -> torch.Tensor:
    """s uniform on the unit sphere: z = 1 - 2 u1, azimuth 2 pi u2."""
    z = 1.0 - 2.0 * u1
    rho = 2.0 * torch.sqrt(u1 * (1.0 - u1))
    phi = 2.0 * math.pi * u2
    return torch.stack([rho * torch.cos(phi), rho * torch.sin(phi), z], dim=-1)


def cosine_direction(n: torch.Tensor, u1: torch.Tensor, u2: torch.Tensor, s_jitter=None) -> torch.Tensor:
    """Cosine-weighted direction about the unit normal n: normalize(n + s).

    The degenerate draw s = -n (probability zero) returns n.  `s_jitter`
    (optional, same shape as s) is added to s by the conditioning probe of
    ``render.float32_sensitivity`` only.
    """
    s = uniform_sphere(u1, u2)
    if s_jitter is not None:
        s = s + s_jitter
    d = n + s
    l2 = (d * d).sum(-1, keepdim=True)
    safe = torch.where(l2 > 1e-20, l2, torch.ones_like(l2))
    return torch.where(l2 > 1e-20, d / torch.sqrt(safe), n.expand_as(d))
