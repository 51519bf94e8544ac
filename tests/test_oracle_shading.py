"""Pins of the oracle's env lookup and BRDF against closed forms and quadrature."""
import math

import numpy as np
import pytest
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


# ---- pins of brdf() itself (Sec. 3.1 simplified Disney model, Sec. 4.1 alpha = r^2,
# Sec. 4.2 height-correlated Smith, Sec. 5 F0 = 0.04) ---------------------------

def _spec(rough, n, wi, wo, f0):
    """brdf()'s specular term: the full value with zero albedo, one channel."""
    z = torch.zeros(*wi.shape[:-1], 3, dtype=torch.float64)
    return shading.brdf(z, rough, n, wi, wo, f0)[..., 0]


def _microfacet_in_angles(alpha, th_i, th_o, dphi, f0):
    """The GGX-Smith microfacet BRDF D F G2 / (4 cos_i cos_o) written in angles (Walter et al. 2007,
    Heitz 2014): D from tan(theta_h), G2 = 1 / (1 + Lambda_i + Lambda_o) with Lambda from tan(theta),
    and w_o.h = cos of half the angle between w_i and w_o."""
    ci, co = np.cos(th_i), np.cos(th_o)
    cos_io = np.sin(th_i) * np.sin(th_o) * np.cos(dphi) + ci * co          # w_i . w_o
    half = 0.5 * np.arccos(np.clip(cos_io, -1.0, 1.0))                     # angle between w_o and h
    voh = np.cos(half)
    cos_h = (ci + co) / (2.0 * voh)                                        # n . h = n.(w_i + w_o) / |w_i + w_o|
    tan2_h = (1.0 - cos_h ** 2) / cos_h ** 2
    d = 1.0 / (np.pi * alpha ** 2 * cos_h ** 4 * (1.0 + tan2_h / alpha ** 2) ** 2)

    def lam(th):
        return 0.5 * (-1.0 + np.sqrt(1.0 + alpha ** 2 * np.tan(th) ** 2))
    g2 = 1.0 / (1.0 + lam(th_i) + lam(th_o))
    f = f0 + (1.0 - f0) * (1.0 - voh) ** 5
    return d * f * g2 / (4.0 * ci * co)


def _dirs(th, ph):
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=-1)


def test_brdf_peak_at_normal_incidence():
    # w_i = w_o = n: D = 1 / (pi alpha^2), F = F0, G2 / (4 NoL NoV) = 1/4, so f_spec = F0 / (4 pi r^4)
    n = torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64)
    for r in (0.09, 0.3, 0.55, 1.0):
        for f0 in (0.0, 0.04, 1.0):
            got = float(_spec(torch.tensor([r], dtype=torch.float64), n, n, n, f0)[0])
            assert got == pytest.approx(f0 / (4.0 * math.pi * r ** 4), rel=1e-10, abs=0.0), (r, f0, got)
    # the diffuse lobe adds albedo / pi on top
    alb = torch.tensor([[0.2, 0.5, 0.9]], dtype=torch.float64)
    full = shading.brdf(alb, torch.tensor([0.5], dtype=torch.float64), n, n, n, 0.04)
    assert torch.allclose(full - alb / math.pi, torch.full_like(full, 0.04 / (4 * math.pi * 0.5 ** 4)), rtol=1e-13)


def test_brdf_matches_the_microfacet_model_in_angles():
    rng = np.random.default_rng(11)
    k = 4000
    th_i, th_o = rng.uniform(0.02, 1.53, k), rng.uniform(0.02, 1.53, k)
    ph_i, ph_o = rng.uniform(-np.pi, np.pi, k), rng.uniform(-np.pi, np.pi, k)
    rough = rng.uniform(0.09, 1.0, k)
    # a random rotation moves the local frame (normal +z) to an arbitrary normal
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    n = np.broadcast_to(q @ np.array([0.0, 0.0, 1.0]), (k, 3))
    wi = _dirs(th_i, ph_i) @ q.T
    wo = _dirs(th_o, ph_o) @ q.T
    for f0 in (0.04, 0.0, 1.0):
        got = _spec(torch.from_numpy(rough), torch.from_numpy(n.copy()), torch.from_numpy(wi), torch.from_numpy(wo),
                    f0).numpy()
        ref = _microfacet_in_angles(rough ** 2, th_i, th_o, ph_i - ph_o, f0)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=0.0)


def test_brdf_directional_albedo_closed_form_at_alpha_one():
    # r = 1, F0 = 1: D = 1/pi and F = 1, and with height-correlated Smith the
    # directional albedo has the closed form E(mu) = 1 - mu ln(1 + 1/mu)
    th = np.linspace(0.0, np.pi / 2, 1201)
    ph = np.linspace(-np.pi, np.pi, 1201)
    T, PH = np.meshgrid(th, ph, indexing="ij")
    wi = torch.from_numpy(_dirs(T, PH))
    n = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64).expand_as(wi)
    one = torch.ones(T.shape, dtype=torch.float64)
    for th_o in (0.0, 0.4, 0.9, 1.3):
        wo = torch.from_numpy(_dirs(np.full_like(T, th_o), np.zeros_like(T)))
        f = _spec(one, n, wi, wo, 1.0).numpy()
        integrand = f * np.cos(T) * np.sin(T)
        e = np.trapezoid(np.trapezoid(integrand, ph, axis=1), th)
        mu = math.cos(th_o)
        assert e == pytest.approx(1.0 - mu * math.log1p(1.0 / mu), abs=2e-5), (th_o, e)


def test_ggx_smith_white_furnace_energy():
    # the energy of the specular lobe (F = 1) at several roughnesses and view angles:
    # quadrature of brdf() against quadrature of the angle form, on the same grid,
    # and bounded by 1 (Smith masking only removes energy)
    th = np.linspace(1e-4, np.pi / 2 - 1e-4, 1601)
    ph = np.linspace(-np.pi, np.pi, 801)
    T, PH = np.meshgrid(th, ph, indexing="ij")
    wi = torch.from_numpy(_dirs(T, PH))
    n = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64).expand_as(wi)
    for r in (0.3, 0.6, 1.0):
        rr = torch.full(T.shape, r, dtype=torch.float64)
        for th_o in (0.1, 0.7, 1.2):
            wo = torch.from_numpy(_dirs(np.full_like(T, th_o), np.zeros_like(T)))
            f = _spec(rr, n, wi, wo, 1.0).numpy()
            g = _microfacet_in_angles(r ** 2, T, np.full_like(T, th_o), PH, 1.0)
            quad = lambda v: np.trapezoid(np.trapezoid(v * np.cos(T) * np.sin(T), ph, axis=1), th)
            e_brdf, e_ref = quad(f), quad(g)
            assert e_brdf == pytest.approx(e_ref, rel=1e-9), (r, th_o)
            assert 0.3 < e_brdf <= 1.0 + 1e-3, (r, th_o, e_brdf)
