"""Multiple importance sampling of the primary directions  (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.1: for every primary point a light-importance ray and a GGX-importance
ray are sampled and combined with Veach's balance heuristic; the GGX rays
come from the distribution of visible normals (Heitz 2018); alpha =
roughness^2.  With n_L light and n_G GGX samples among the N directions of a
point the balance-heuristic estimator of Eq. 1 is

    L(x, w_o) = sum_i f_r(w_i, w_o) (n . w_i)+ L(x, w_i) / (n_L p_L(w_i) + n_G p_G(w_i)).

Readings:
  * sample i uses the light strategy for even i and GGX for odd i, so
    n_G = floor(N / 2) and n_L = N - n_G; a point seen from below (n . w_o
    <= 1e-4) has no visible normals, so all its samples are light samples
    (n_G = 0);
  * the light distribution picks a texel of the bound environment map with
    probability proportional to its luminance 0.2126 R + 0.7152 G + 0.0722 B
    (negative parts clipped, plus 1e-6 so that every texel can be drawn),
    then a point uniform in (phi, theta) inside the texel, whose solid-angle
    density is p_texel / (dphi dtheta sin(theta)).  The texel follows the
    lookup's convention: column c spans phi in [2 pi c / W - pi, ...), row r
    spans theta in [pi r / H, ...);
  * the texel is found by inverting a marginal (rows) and a conditional
    (columns) CDF with the two uniforms of the sample; the residual of each
    inversion is the position inside the texel.  Those CDFs decide integers
    from floating point, so they are built in float32 exactly as the kernel
    builds them: products and sums rounded one at a time (no fused
    multiply-add), running sums in index order, each normalised by its
    total with one float32 division, the last entry set to 1;
  * GGX visible-normal sampling in the frame of Duff et al. (2017) about
    the primary normal;  p_G(w) = G1(w_o) D(h) / (4 n . w_o) with h the half
    vector, G1 Smith's term and D the GGX distribution with alpha^2 = r^4
    (zero where w_o . h <= 0 or n . h <= 0);
  * the secondary directions at x' stay cosine-weighted (the supplementary
    casts "8 random rays via stratified sampling" there).

Pins (tests/test_oracle_mis.py): both densities integrate to 1 over the
sphere; texel frequencies of the light sampler match its probabilities and
positions are uniform inside a texel; E[p_cos / p_G] = 1 for GGX samples;
the mirror limit of the GGX sampler; the furnace test and agreement with
cosine sampling for the balance-heuristic estimator.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import shading

LUMA32 = np.array([0.2126, 0.7152, 0.0722], np.float32)
LUM_FLOOR32 = np.float32(1e-6)
NOV_MIN = 1e-4


def env_cdf(env: np.ndarray):
    """(marginal [H + 1], conditional [H, W + 1]) float32 CDFs of the texel distribution."""
    e = np.asarray(env, np.float32)
    H, W = e.shape[0], e.shape[1]
    lum = (e[..., 0] * LUMA32[0] + e[..., 1] * LUMA32[1]) + e[..., 2] * LUMA32[2]   # each op rounded
    lum = np.maximum(lum, np.float32(0.0)) + LUM_FLOOR32
    cond = np.zeros((H, W + 1), np.float32)
    totals = np.zeros(H, np.float32)
    for r in range(H):
        run = np.cumsum(lum[r], dtype=np.float32)          # sequential float32 running sums
        totals[r] = run[-1]
        cond[r, 1:] = run / run[-1]
        cond[r, W] = np.float32(1.0)
    marg = np.zeros(H + 1, np.float32)
    run = np.cumsum(totals, dtype=np.float32)
    marg[1:] = run / run[-1]
    marg[H] = np.float32(1.0)
    return marg, cond


def _invert(cdf: np.ndarray, u: np.ndarray):
    """Index k with cdf[k] <= u < cdf[k + 1] and the residual (u - cdf[k]) / (cdf[k + 1] - cdf[k])."""
    k = np.searchsorted(cdf, u, side="right") - 1
    k = np.clip(k, 0, cdf.shape[-1] - 2)
    lo = cdf[k].astype(np.float64)
    hi = cdf[k + 1].astype(np.float64)
    return k, (u - lo) / (hi - lo)


def sample_light(u1, u2, marg, cond) -> torch.Tensor:
    """Directions [..., 3] drawn from the texel distribution (u1 picks the row, u2 the column)."""
    u1 = np.asarray(u1, np.float64)
    u2 = np.asarray(u2, np.float64)
    H, W = cond.shape[0], cond.shape[1] - 1
    r, ur = _invert(marg, u1)
    c = np.empty_like(r)
    uc = np.empty_like(u2)
    for row in np.unique(r):
        m = r == row
        c[m], uc[m] = _invert(cond[row], u2[m])
    theta = math.pi * (r + ur) / H
    phi = 2.0 * math.pi * (c + uc) / W - math.pi
    st = np.sin(theta)
    return torch.from_numpy(np.stack([st * np.cos(phi), st * np.sin(phi), np.cos(theta)], axis=-1))


def pdf_light(w: torch.Tensor, marg, cond) -> torch.Tensor:
    """Solid-angle density of sample_light at directions w [..., 3]."""
    H, W = cond.shape[0], cond.shape[1] - 1
    x, y, z = w[..., 0], w[..., 1], w[..., 2]
    theta = torch.acos(z.clamp(-1.0, 1.0))
    phi = torch.atan2(y, x)
    r = torch.clamp(torch.floor(theta / math.pi * H).to(torch.int64), 0, H - 1)
    c = torch.clamp(torch.floor((phi + math.pi) / (2.0 * math.pi) * W).to(torch.int64), 0, W - 1)
    m = torch.from_numpy(marg.astype(np.float64))
    cd = torch.from_numpy(cond.astype(np.float64))
    p_t = (m[r + 1] - m[r]) * (cd[r, c + 1] - cd[r, c])
    sin_t = torch.sqrt(x * x + y * y)
    return p_t / ((2.0 * math.pi / W) * (math.pi / H) * sin_t)


def pdf_light_neighbours(w: torch.Tensor, marg, cond, delta: float):
    """Largest |p_L(w) - p_L'(w)| over the texels adjacent to w's own across a boundary that w lies
    within `delta` radians of (0 elsewhere): the densities a kernel could use for w after rounding."""
    H, W = cond.shape[0], cond.shape[1] - 1
    x, y, z = w[..., 0], w[..., 1], w[..., 2]
    theta = torch.acos(z.clamp(-1.0, 1.0))
    phi = torch.atan2(y, x)
    tq = theta / math.pi * H
    tp = (phi + math.pi) / (2.0 * math.pi) * W
    r = torch.clamp(torch.floor(tq).to(torch.int64), 0, H - 1)
    c = torch.clamp(torch.floor(tp).to(torch.int64), 0, W - 1)
    m = torch.from_numpy(marg.astype(np.float64))
    cd = torch.from_numpy(cond.astype(np.float64))
    sin_t = torch.sqrt(x * x + y * y)
    scale = (2.0 * math.pi / W) * (math.pi / H) * sin_t

    def p_at(rr, cc):
        return (m[rr + 1] - m[rr]) * (cd[rr, cc + 1] - cd[rr, cc]) / scale
    base = p_at(r, c)
    worst = torch.zeros_like(base)
    dq = delta * H / math.pi
    dp = delta * W / (2.0 * math.pi)
    for near, rr, cc in ((tq - r < dq, torch.clamp(r - 1, 0, H - 1), c),
                         (r + 1 - tq < dq, torch.clamp(r + 1, 0, H - 1), c),
                         (tp - c < dp, r, torch.remainder(c - 1, W)),
                         (c + 1 - tp < dp, r, torch.remainder(c + 1, W))):
        worst = torch.where(near, torch.maximum(worst, (p_at(rr, cc) - base).abs()), worst)
    return worst


def frame(n: torch.Tensor):
    """Orthonormal (t, b) completing the unit normal n (Duff et al. 2017)."""
    sign = torch.where(n[..., 2] >= 0, torch.ones_like(n[..., 2]), -torch.ones_like(n[..., 2]))
    a = -1.0 / (sign + n[..., 2])
    b = n[..., 0] * n[..., 1] * a
    t = torch.stack([1.0 + sign * n[..., 0] ** 2 * a, sign * b, -sign * n[..., 0]], dim=-1)
    bt = torch.stack([b, sign + n[..., 1] ** 2 * a, -n[..., 1]], dim=-1)
    return t, bt


def sample_ggx(n: torch.Tensor, wo: torch.Tensor, alpha: torch.Tensor, u1, u2) -> torch.Tensor:
    """Directions [..., 3] reflected about GGX visible normals (Heitz 2018) seen from wo."""
    u1 = torch.as_tensor(np.asarray(u1, np.float64))
    u2 = torch.as_tensor(np.asarray(u2, np.float64))
    t, bt = frame(n)
    v = torch.stack([(wo * t).sum(-1), (wo * bt).sum(-1), (wo * n).sum(-1)], dim=-1)
    vh = torch.stack([alpha * v[..., 0], alpha * v[..., 1], v[..., 2]], dim=-1)
    vh = vh / vh.norm(dim=-1, keepdim=True)
    lensq = vh[..., 0] ** 2 + vh[..., 1] ** 2
    inv = torch.where(lensq > 0, 1.0 / torch.sqrt(torch.where(lensq > 0, lensq, torch.ones_like(lensq))),
                      torch.zeros_like(lensq))
    t1 = torch.where((lensq > 0)[..., None], torch.stack([-vh[..., 1] * inv, vh[..., 0] * inv,
                                                          torch.zeros_like(inv)], -1),
                     torch.tensor([1.0, 0.0, 0.0], dtype=vh.dtype).expand_as(vh))
    t2 = torch.cross(vh, t1, dim=-1)
    rr = torch.sqrt(u1)
    ph = 2.0 * math.pi * u2
    p1 = rr * torch.cos(ph)
    p2 = rr * torch.sin(ph)
    s = 0.5 * (1.0 + vh[..., 2])
    p2 = (1.0 - s) * torch.sqrt(1.0 - p1 * p1) + s * p2
    nh = p1[..., None] * t1 + p2[..., None] * t2 + \
        torch.sqrt(torch.clamp(1.0 - p1 * p1 - p2 * p2, min=0.0))[..., None] * vh
    ne = torch.stack([alpha * nh[..., 0], alpha * nh[..., 1], torch.clamp(nh[..., 2], min=0.0)], dim=-1)
    ne = ne / ne.norm(dim=-1, keepdim=True)
    h = ne[..., 0:1] * t + ne[..., 1:2] * bt + ne[..., 2:3] * n
    return 2.0 * (wo * h).sum(-1, keepdim=True) * h - wo


def pdf_ggx(w: torch.Tensor, n: torch.Tensor, wo: torch.Tensor, alpha: torch.Tensor) -> torch.Tensor:
    """Solid-angle density of sample_ggx: G1(w_o) D(h) / (4 n . w_o)."""
    nov = (n * wo).sum(-1)
    hv = w + wo
    hl = hv.norm(dim=-1)
    h = hv / torch.where(hl > 0, hl, torch.ones_like(hl))[..., None]
    noh = (n * h).sum(-1)
    voh = (wo * h).sum(-1)
    a2 = alpha * alpha
    d = shading.ggx_d(torch.clamp(noh, min=0.0), a2)
    nov_c = torch.clamp(nov, min=NOV_MIN)
    g1 = 2.0 * nov_c / (nov_c + torch.sqrt(a2 + (1.0 - a2) * nov_c * nov_c))
    ok = (nov > NOV_MIN) & (noh > 0) & (voh > 0) & (hl > 0)
    return torch.where(ok, g1 * d / (4.0 * nov_c), torch.zeros_like(d))


def primary_directions(n, wo, rough, u1, u2, n_dirs: int, marg, cond):
    """MIS directions w [P, N, 3] and their Eq. 1 factors (n . w)+ / (n_L p_L + n_G p_G) [P, N].

    n, wo [P, 3]; rough [P]; u1, u2 [P, N] (the slot-0 uniforms of each sample).
    """
    P, N = u1.shape
    alpha = (rough * rough)[:, None].expand(P, N)
    nv = n[:, None, :].expand(P, N, 3)
    wv = wo[:, None, :].expand(P, N, 3)
    ggx_ok = (n * wo).sum(-1) > NOV_MIN                            # [P]
    use_g = ggx_ok[:, None] & torch.from_numpy((np.arange(N) % 2 == 1)[None, :])
    w_l = sample_light(u1.numpy(), u2.numpy(), marg, cond)
    w_g = sample_ggx(nv, wv, alpha, u1, u2)
    w = torch.where(use_g[..., None], w_g, w_l)
    n_g = torch.where(ggx_ok, torch.full_like(alpha[:, 0], N // 2), torch.zeros_like(alpha[:, 0]))[:, None]
    n_l = N - n_g
    den = n_l * pdf_light(w, marg, cond) + n_g * pdf_ggx(w, nv, wv, alpha)
    cos = torch.clamp((nv * w).sum(-1), min=0.0)
    return w, cos / den
