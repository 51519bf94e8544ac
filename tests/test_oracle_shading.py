"""Pins of the oracle's env lookup and BRDF against closed forms and quadrature."""
import math

import numpy as np
import torch

from oracle import shading


def _dir(theta, phi):
    return torch.stack([torch.sin(theta) * torch.cos(phi), torch.sin(theta) * torch.sin(phi),
                        torch.cos(theta)], dim=-1)


def test_env_constant_map():
    env = torch.zeros(8, 16, 4, dtype=torch.float64)
    env[..., :3] = torch.tensor([0.25, 2.0, 7.0], dtype=torch.float64)
    w = torch.from_numpy(np.random.default_rng(0).normal(size=(1000, 3)))
    w = w / w.norm(dim=1, keepdim=True)
    out = shading.env_lookup(env, w)
    assert torch.allclose(out, env[0, 0, :3].expand(1000, 3), atol=1e-14)


def test_env_texel_centres_are_exact():
    H, W = 6, 12
    env = torch.from_numpy(np.random.default_rng(1).lognormal(size=(H, W, 4)))
    r, c = torch.meshgrid(torch.arange(H), torch.arange(W), indexing="ij")
    theta = (r.double() + 0.5) / H * math.pi
    phi = (c.double() + 0.5) / W * 2 * math.pi - math.pi
    out = shading.env_lookup(env, _dir(theta, phi))
    assert torch.allclose(out, env[..., :3], atol=1e-12)


def test_env_linear_in_azimuth_and_seam():
    H, W = 4, 10
    env = torch.zeros(H, W, 4, dtype=torch.float64)
    env[..., 0] = torch.arange(W, dtype=torch.float64)[None, :]
    phi = torch.linspace(-math.pi + 0.5 * 2 * math.pi / W, math.pi - 0.5 * 2 * math.pi / W, 101,
                         dtype=torch.float64)
    theta = torch.full_like(phi, 1.0)
    s = (phi + math.pi) / (2 * math.pi) * W - 0.5
    out = shading.env_lookup(env, _dir(theta, phi))[:, 0]
    assert torch.allclose(out, s, atol=1e-12)
    # across the seam the map interpolates between the last and the first column
    eps = 1e-9
    a = shading.env_lookup(env, _dir(torch.tensor([1.0], dtype=torch.float64), torch.tensor([math.pi - eps], dtype=torch.float64)))[0, 0]
    b = shading.env_lookup(env, _dir(torch.tensor([1.0], dtype=torch.float64), torch.tensor([-math.pi + eps], dtype=torch.float64)))[0, 0]
    assert abs(float(a) - (W - 1) / 2) < 1e-6 and abs(float(b) - (W - 1) / 2) < 1e-6


def test_ggx_d_is_normalised():
    # integral over the hemisphere of D(h) (n.h) dw_h = 1
    th = torch.linspace(0, math.pi / 2, 200001, dtype=torch.float64)
    for rough in [0.09, 0.3, 0.7, 1.0]:
        a2 = torch.tensor((rough * rough) ** 2, dtype=torch.float64)
        integrand = shading.ggx_d(torch.cos(th), a2) * torch.cos(th) * torch.sin(th)
        val = 2 * math.pi * torch.trapezoid(integrand, th)
        assert abs(float(val) - 1.0) < 2e-4, (rough, float(val))


def test_smith_vis_equals_textbook_g2():
    rng = np.random.default_rng(2)
    nol = torch.from_numpy(rng.uniform(1e-3, 1, 1000))
    nov = torch.from_numpy(rng.uniform(1e-3, 1, 1000))
    alpha = torch.from_numpy(rng.uniform(0.0081, 1, 1000))
    a2 = alpha * alpha

    def lam(mu):
        tan2 = (1 - mu * mu) / (mu * mu)
        return (-1 + torch.sqrt(1 + a2 * tan2)) / 2

    g2 = 1.0 / (1.0 + lam(nol) + lam(nov))
    assert torch.allclose(shading.smith_vis(nol, nov, a2), g2 / (4 * nol * nov), rtol=1e-12)


def test_schlick_end_points():
    assert float(shading.schlick_fresnel(torch.tensor(1.0, dtype=torch.float64), 0.04)) == 0.04
    assert float(shading.schlick_fresnel(torch.tensor(0.0, dtype=torch.float64), 0.04)) == 1.0


def test_brdf_lambert_and_reciprocity():
    rng = np.random.default_rng(3)
    n = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64).expand(500, 3)

    def hemi(k):
        v = torch.from_numpy(rng.normal(size=(k, 3)))
        v[:, 2] = v[:, 2].abs() + 0.05
        return v / v.norm(dim=1, keepdim=True)

    wi, wo = hemi(500), hemi(500)
    alb = torch.from_numpy(rng.uniform(0, 1, (500, 3)))
    r = torch.from_numpy(rng.uniform(0.09, 1, 500))
    lam = shading.brdf(alb, r, n, wi, wo, lambert=True)
    assert torch.allclose(lam, alb / math.pi)
    # with both directions above the surface (and NoV > 1e-4) the BRDF is reciprocal
    assert torch.allclose(shading.brdf(alb, r, n, wi, wo), shading.brdf(alb, r, n, wo, wi), rtol=1e-12)
