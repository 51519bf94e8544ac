"""Stage (e): environment lighting, BRDF and the Monte Carlo sums  (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Environment map (Sec. 2.2): an equirectangular map whose texels act as
point lights; the incoming radiance L_i is interpolated from its pixels.
Reading (the paper gives no convention): phi = atan2(w_y, w_x), theta =
acos(w_z); texel coordinates s = (phi + pi) / (2 pi) * W - 1/2 and
q = theta / pi * H - 1/2; bilinear interpolation, wrapping in s and
clamping in q.  The map is continuous across the phi = +-pi seam.

BRDF (Sec. 3.1 "simplified Disney model"; Sec. 4.1; Sec. 4.2 teacher; Sec. 5):
  f_r = a / pi + D * F * Vis, with
  alpha = r^2 (the remap of Sec. 4.1),
  D   = alpha^2 / (pi ((n.h)^2 (alpha^2 - 1) + 1)^2)          (GGX),
  F   = F0 + (1 - F0)(1 - w_o.h)^5, F0 = 0.04                (Schlick; Sec. 4.2, Sec. 5),
  Vis = 0.5 / (NoL sqrt(NoV^2 (1 - alpha^2) + alpha^2)
               + NoV sqrt(NoL^2 (1 - alpha^2) + alpha^2))     (height-correlated Smith),
  NoL = max(n.w_i, 0), NoV = max(n.w_o, 1e-4), n.h clamped at 0.
Readings: no normal flipping; the specular term is grey (F0 scalar);
h = (w_i + w_o)/|w_i + w_o| with w_o.h = |w_i + w_o| / 2; a degenerate
half vector (|w_i + w_o|^2 <= 1e-20) gives n.h = 0.  Every direction and
normal reaching brdf() is a unit vector in float64 (render.py normalises
the G-buffer's n and w_o, B's n' and the sampled directions), so D is the
textbook form above.

Monte Carlo sums with cosine-weighted directions, p(w) = (w.n) / pi, so the
cosine over the pdf in Eq. 1 is pi:
  secondary (Eq. 1 at x'_i, only the outgoing direction -w_i):
      L'_o,i = (pi / M) sum_j v'_ij L_env(w'_ij) f_r(a', r', n'; w'_ij, -w_i)
  incoming radiance (Eq. 2, soft V):
      L(x, w_i) = v_i L_env(w_i) + (1 - v_i) L'_o,i
  primary (Eq. 1):
      L(x, w_o) = (pi / N) sum_i L(x, w_i) f_r(a, r, n; w_i, w_o)

Pins (tests/test_oracle_shading.py): constant and linear env maps, exact
texel centres and seam continuity; D integrates to 1 against n.h over the
sphere (quadrature); Vis equals the textbook height-correlated
G2 = 1 / (1 + Lambda(w_o) + Lambda(w_i)) divided by 4 NoL NoV; Schlick's end
points; and brdf() itself: its peak F0 / (4 pi alpha^2) at normal incidence,
agreement with the microfacet model written in angles (D from tan theta_h,
G2 from Lambda, w_o.h from half the angle between w_i and w_o), the closed-
form directional albedo 1 - mu ln(1 + 1/mu) of the alpha = 1, F = 1 lobe,
and the white-furnace energy of the GGX-Smith lobe against quadrature of
that angle form; the white furnace of the whole estimator (render tests).
"""
from __future__ import annotations

import math

import torch

F0_DEFAULT = 0.04


def env_lookup(env: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """Bilinearly interpolated radiance of env [H, W, C>=3] in directions w [..., 3]."""
    h, wd = env.shape[0], env.shape[1]
    phi = torch.atan2(w[..., 1], w[..., 0])
    theta = torch.acos(w[..., 2].clamp(-1.0, 1.0))
    s = (phi + math.pi) / (2.0 * math.pi) * wd - 0.5
    q = theta / math.pi * h - 0.5
    s0 = torch.floor(s)
    q0 = torch.floor(q)
    fs = (s - s0)[..., None]
    fq = (q - q0)[..., None]
    s0 = s0.to(torch.int64)
    q0 = q0.to(torch.int64)
    c0 = torch.remainder(s0, wd)
    c1 = torch.remainder(s0 + 1, wd)
    r0 = q0.clamp(0, h - 1)
    r1 = (q0 + 1).clamp(0, h - 1)
    e = env[..., :3].to(torch.float64)
    top = (1.0 - fs) * e[r0, c0] + fs * e[r0, c1]
    bot = (1.0 - fs) * e[r1, c0] + fs * e[r1, c1]
    return (1.0 - fq) * top + fq * bot


def ggx_d(noh: torch.Tensor, a2: torch.Tensor) -> torch.Tensor:
    """GGX normal distribution D(h) = a2 / (pi ((n.h)^2 (a2 - 1) + 1)^2), alpha^2 = a2, unit vectors."""
    return a2 / (math.pi * (noh * noh * (a2 - 1.0) + 1.0) ** 2)


def schlick_fresnel(voh: torch.Tensor, f0: float) -> torch.Tensor:
    """F = F0 + (1 - F0)(1 - w_o.h)^5."""
    return f0 + (1.0 - f0) * (1.0 - voh) ** 5


def smith_vis(nol: torch.Tensor, nov: torch.Tensor, a2: torch.Tensor) -> torch.Tensor:
    """Height-correlated Smith G2 / (4 NoL NoV), in the form that needs no division by NoL."""
    return 0.5 / (nol * torch.sqrt(nov * nov * (1.0 - a2) + a2)
                  + nov * torch.sqrt(nol * nol * (1.0 - a2) + a2))


def brdf(albedo: torch.Tensor, rough: torch.Tensor, n: torch.Tensor, wi: torch.Tensor,
         wo: torch.Tensor, f0: float = F0_DEFAULT, lambert: bool = False) -> torch.Tensor:
    """f_r(a, r, n; w_i, w_o) [..., 3] with the simplified Disney model above.

    albedo, n, wi, wo carry a trailing axis of 3; rough has the shape of the
    direction axes alone (it broadcasts against n.w_i).
    """
    diffuse = albedo / math.pi
    if lambert:
        return diffuse.expand(*torch.broadcast_shapes(diffuse.shape, wi.shape))
    alpha = rough * rough
    a2 = alpha * alpha
    nol = (n * wi).sum(-1).clamp(min=0.0)
    nov = (n * wo).sum(-1).clamp(min=1e-4)
    hv = wi + wo
    hl2 = (hv * hv).sum(-1)
    ok = hl2 > 1e-20
    hl = torch.sqrt(torch.where(ok, hl2, torch.ones_like(hl2)))
    h = hv / hl[..., None]
    # n.h clamped at 0 (D = a2 / pi there); a degenerate half vector gives n.h = 0 and w_o.h = 0
    noh = torch.where(ok, (n * h).sum(-1), torch.zeros_like(hl)).clamp(min=0.0)
    voh = torch.where(ok, 0.5 * hl, torch.zeros_like(hl))
    spec = ggx_d(noh, a2) * schlick_fresnel(voh, f0) * smith_vis(nol, nov, a2)
    return diffuse + spec[..., None]


def mc_sum(weights: torch.Tensor, count: int) -> torch.Tensor:
    """(pi / count) * sum over the direction axis (-2) of per-direction terms [..., K, 3]."""
    return (math.pi / count) * weights.sum(dim=-2)
