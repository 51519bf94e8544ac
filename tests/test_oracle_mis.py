"""Pins of the oracle's multiple importance sampling of the primary directions (Sec. 4.1)."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import scenegen
from oracle import mis, render, sampling, shading


def _env(h=6, w=10, seed=0):
    rng = np.random.default_rng(seed)
    e = np.ones((h, w, 4), np.float32)
    e[..., :3] = rng.lognormal(0.0, 1.5, (h, w, 3)).astype(np.float32)
    return e


def _sphere_grid(nt=720, nphi=1440):
    # midpoints in (theta, phi); each light texel is split into whole cells when nt, nphi are multiples of H, W
    t = (np.arange(nt) + 0.5) * math.pi / nt
    p = (np.arange(nphi) + 0.5) * 2.0 * math.pi / nphi - math.pi
    T, Ph = np.meshgrid(t, p, indexing="ij")
    w = np.stack([np.sin(T) * np.cos(Ph), np.sin(T) * np.sin(Ph), np.cos(T)], -1)
    dA = np.sin(T) * (math.pi / nt) * (2.0 * math.pi / nphi)
    return torch.from_numpy(w), dA


def test_light_density_integrates_to_one():
    marg, cond = mis.env_cdf(_env())
    w, dA = _sphere_grid()
    p = mis.pdf_light(w, marg, cond).numpy()
    assert float((p * dA).sum()) == pytest.approx(1.0, abs=1e-9)


def test_light_sampler_picks_texels_with_their_probability_and_fills_them_uniformly():
    env = _env(4, 8, 1)
    marg, cond = mis.env_cdf(env)
    rng = np.random.default_rng(2)
    n = 400_000
    u1 = np.floor(rng.random(n) * 2 ** 24) * 2.0 ** -24    # the kernel's 24-bit uniforms
    u2 = np.floor(rng.random(n) * 2 ** 24) * 2.0 ** -24
    w = mis.sample_light(u1, u2, marg, cond).numpy()
    theta = np.arccos(np.clip(w[:, 2], -1, 1))
    phi = np.arctan2(w[:, 1], w[:, 0])
    r = np.clip(np.floor(theta / math.pi * 4).astype(int), 0, 3)
    c = np.clip(np.floor((phi + math.pi) / (2 * math.pi) * 8).astype(int), 0, 7)
    p_t = np.diff(marg.astype(np.float64))[:, None] * np.diff(cond.astype(np.float64), axis=1)
    counts = np.zeros((4, 8))
    np.add.at(counts, (r, c), 1)
    z = (counts - n * p_t) / np.sqrt(n * p_t * (1 - p_t))
    assert np.abs(z).max() < 5.0
    # inside a texel the position is uniform in (phi, theta): fractional parts average 1/2
    fr = theta / math.pi * 4 - r
    assert abs(fr.mean() - 0.5) < 0.01 and abs(((phi + math.pi) / (2 * math.pi) * 8 - c).mean() - 0.5) < 0.01
    # the texel probabilities are proportional to the clipped luminance (plus the floor)
    lum = env[..., :3].astype(np.float64) @ np.array([0.2126, 0.7152, 0.0722]) + 1e-6
    np.testing.assert_allclose(p_t, lum / lum.sum(), rtol=1e-5)


@pytest.mark.parametrize("alpha, view_deg", [(0.5, 30.0), (0.2, 70.0)])
def test_ggx_density_integrates_to_one(alpha, view_deg):
    w, dA = _sphere_grid(1440, 2880)
    n = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64).expand_as(w)
    v = math.radians(view_deg)
    wo = torch.tensor([math.sin(v), 0.0, math.cos(v)], dtype=torch.float64).expand_as(w)
    p = mis.pdf_ggx(w, n, wo, torch.full(w.shape[:-1], alpha, dtype=torch.float64)).numpy()
    assert float((p * dA).sum()) == pytest.approx(1.0, abs=4e-3)


def _rand_unit(rng, k):
    v = rng.normal(size=(k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_ggx_sampler_follows_its_density():
    # E[p_cos(w) / p_G(w)] over GGX samples is the cosine density's mass on the sampler's
    # support, the upper hemisphere: 1
    rng = np.random.default_rng(3)
    k = 200_000
    n = torch.from_numpy(_rand_unit(rng, 1)).expand(k, 3)
    wo = torch.from_numpy(_rand_unit(rng, 1))
    if float((n[0] * wo[0]).sum()) < 0.2:
        wo = -wo if float((n[0] * wo[0]).sum()) < 0 else (wo + n[:1]) / (wo + n[:1]).norm()
    wo = wo.expand(k, 3)
    alpha = torch.full((k,), 0.35, dtype=torch.float64)
    w = mis.sample_ggx(n, wo, alpha, rng.random(k), rng.random(k))
    cos = (n * w).sum(-1)
    p = mis.pdf_ggx(w, n, wo, alpha)
    ok = (cos > 0) & (p > 0)
    ratio = torch.where(ok, (cos / math.pi) / torch.where(ok, p, torch.ones_like(p)), torch.zeros_like(p)).numpy()
    assert abs(ratio.mean() - 1.0) < 5.0 * ratio.std() / math.sqrt(k)
    np.testing.assert_allclose(w.norm(dim=-1).numpy(), 1.0, atol=1e-12)


def test_ggx_mirror_limit():
    rng = np.random.default_rng(4)
    n = torch.from_numpy(_rand_unit(rng, 64))
    wo = torch.from_numpy(_rand_unit(rng, 64))
    wo = torch.where(((n * wo).sum(-1) < 0)[:, None], -wo, wo)
    w = mis.sample_ggx(n, wo, torch.full((64,), 1e-6, dtype=torch.float64), rng.random(64), rng.random(64))
    mirror = 2.0 * (n * wo).sum(-1, keepdim=True) * n - wo
    assert float((w - mirror).norm(dim=-1).max()) < 1e-4


SMALL = scenegen.SceneConfig("small", 3, 2, 4096, m_dirs=1, levels=4, log2_T=10, base_res=4, max_res=32,
                             env_h=8, env_w=16)


def _scene(env_rgb=None, seed=0):
    sc = scenegen.make_scene(SMALL, seed)
    env = sc.env.copy()
    if env_rgb is not None:
        env[..., :3] = env_rgb
    gb = scenegen.make_gbuffer(SMALL.n_pixels, seed)
    gb["view"][:, :3] = np.where((gb["view"][:, :3] * gb["normal"][:, :3]).sum(1, keepdims=True) < 0,
                                 -gb["view"][:, :3], gb["view"][:, :3])      # mostly front-facing views
    return gb, render.Params.from_arrays(sc.table, sc.brdf, sc.irt, env)


def test_mis_furnace():
    # white environment, V = 1, Lambert: the balance-heuristic estimate converges to the albedo
    gb, prm = _scene(env_rgb=1.0)
    out = render.render(gb, prm, render.Options.from_config(SMALL, sampling="mis", force_vis=1.0, lambert=True))
    np.testing.assert_allclose(out, gb["albedo_rough"][:, :3], rtol=0.03)


def test_mis_matches_the_direct_light_integral():
    # V = 1 makes the radiance the direct-light integral  int f_r Lenv (n . w)+ dw, which a fine
    # sphere quadrature evaluates deterministically; the balance-heuristic estimate converges to it,
    # including a sharp (r = 0.28) lobe seen at a grazing angle, where cosine sampling is still far off
    gb, prm = _scene(seed=1)
    out = render.render(gb, prm, render.Options.from_config(SMALL, force_vis=1.0, sampling="mis"))
    w, dA = _sphere_grid(1440, 2880)
    le = shading.env_lookup(prm.env, w)
    for p in range(SMALL.n_pixels):
        n = torch.from_numpy(gb["normal"][p, :3].astype(np.float64))
        wo = torch.from_numpy(gb["view"][p, :3].astype(np.float64))
        ar = gb["albedo_rough"][p].astype(np.float64)
        fr = shading.brdf(torch.from_numpy(ar[:3]), torch.tensor(ar[3]), n, w, wo)
        cos = torch.clamp((w * n).sum(-1), min=0.0)
        ref = ((fr * le * cos[..., None]).numpy() * dA[..., None]).sum((0, 1))
        np.testing.assert_allclose(out[p], ref, rtol=0.03)


def test_texel_edge_allowance_is_the_neighbouring_density():
    # a direction just inside a column edge: the allowance is |p_L(next texel) - p_L(own texel)|;
    # away from every edge it is 0
    marg, cond = mis.env_cdf(_env(6, 10, 5))
    th = math.pi * 2.5 / 6                       # mid-row 2
    def d(phi):
        return torch.tensor([[math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th)]],
                            dtype=torch.float64)
    edge = 2.0 * math.pi * 4 / 10 - math.pi      # left edge of column 4
    w_in, w_out = d(edge + 1e-7), d(edge - 1e-7)
    got = mis.pdf_light_neighbours(w_in, marg, cond, 1e-6)
    ref = (mis.pdf_light(w_out, marg, cond) - mis.pdf_light(w_in, marg, cond)).abs()
    assert float(got) == pytest.approx(float(ref), rel=1e-6)
    assert float(mis.pdf_light_neighbours(d(edge + 0.1), marg, cond, 1e-6)) == 0.0
