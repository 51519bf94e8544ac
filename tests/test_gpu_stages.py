"""Stage-by-stage parity of the CUDA kernels with the FP64 oracle (through the C ABI)."""
import math

import numpy as np
import pytest
import torch

import scenegen
from oracle import hashgrid, mlp, sampling, shading
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2409_10327_gb300 import build
    build.build()
    from paper_2409_10327_gb300 import binding
    return binding


def _points(P, seed):
    rng = np.random.default_rng(seed)
    pos = np.zeros((P, 4), np.float32)
    pos[:, :3] = rng.uniform(-1.3, 1.3, (P, 3))
    # exact lattice vertices of the 16- and 256-resolution levels, and the box faces
    pos[:64, :3] = (2.0 * rng.integers(0, 17, (64, 3)) / 16 - 1.0)
    pos[64:128, :3] = (2.0 * rng.integers(0, 257, (64, 3)) / 256 - 1.0)
    pos[128:136, :3] = np.array([[1, 1, 1], [-1, -1, -1], [1, -1, 1], [0, 0, 0]] * 2, np.float32)
    return pos


def _full_points(P, seed):
    pos = _points(P, seed)
    rng = np.random.default_rng(seed + 100)
    # exact vertices of the finest (2048) lattice and points a float32 ulp either side of them
    v = (2.0 * rng.integers(0, 2049, (256, 3)) / 2048 - 1.0).astype(np.float32)
    pos[136:392, :3] = v
    pos[392:648, :3] = np.nextafter(v, np.float32(2.0))
    pos[648:904, :3] = np.nextafter(v, np.float32(-2.0))
    return pos


@pytest.mark.parametrize("workload", ["small", "frame800", "serve1080"])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_encode_indices_bit_exact(lib, precision, workload):
    # small: L=8, T=2^14, 16..256; frame800: L=16, T=2^19, 16..2048 (the benchmarked grid);
    # serve1080: L=16, T=2^20, 16..2048 (the batched-serving grid)
    if workload == "small":
        cfg = helpers.small_cfg(precision=precision)
        pos = _points(3001, 1)
    else:
        import dataclasses
        cfg = dataclasses.replace(scenegen.CONFIGS[workload], precision=precision)
        pos = _full_points(20001, 2)
    sc = scenegen.make_scene(cfg, 0)
    r = helpers.renderer_for(cfg, sc)
    feat, idx, w = r.encode(torch.from_numpy(pos).cuda(), want_aux=True)
    res = hashgrid.level_resolutions(cfg.levels, cfg.base_res, cfg.max_res)
    dense = hashgrid.dense_levels(res, 1 << cfg.log2_T)
    table = sc.table.astype(np.float16).astype(np.float64) if precision == "bf16" else sc.table.astype(np.float64)
    f_ref, i_ref, w_ref = hashgrid.encode(torch.from_numpy(pos[:, :3].astype(np.float64)), torch.from_numpy(table),
                                          res, dense, fp32_grid=True, return_aux=True)
    np.testing.assert_array_equal(idx.cpu().numpy().astype(np.int64), i_ref.numpy())
    np.testing.assert_allclose(w.cpu().numpy(), w_ref.numpy(), rtol=0, atol=2e-7)
    np.testing.assert_allclose(feat.cpu().numpy(), f_ref.numpy(), rtol=0, atol=2e-7)


def test_encode_empty_and_ragged(lib):
    cfg = helpers.small_cfg()
    r = helpers.renderer_for(cfg, scenegen.make_scene(cfg, 0))
    f = r.encode(torch.zeros(0, 4, device="cuda"))
    assert f.shape == (0, cfg.levels * 2)
    pos = _points(137, 3)
    f1 = r.encode(torch.from_numpy(pos).cuda())
    f2 = r.encode(torch.from_numpy(pos[:1]).cuda())
    np.testing.assert_array_equal(f1[:1].cpu().numpy(), f2.cpu().numpy())


def test_decode_matches_oracle(lib):
    cfg = helpers.small_cfg(levels=5)
    sc = scenegen.make_scene(cfg, 4, bias_scale=0.3)
    r = helpers.renderer_for(cfg, sc)
    feat = np.random.default_rng(5).normal(0, 0.3, (1000, 10)).astype(np.float32)
    out = r.decode(torch.from_numpy(feat).cuda()).cpu().numpy()
    a, rr, n = mlp.brdf_decoder(torch.from_numpy(feat.astype(np.float64)), mlp.as_layers(sc.brdf))
    np.testing.assert_allclose(out[:, 0:3], n.numpy(), atol=2e-6)
    np.testing.assert_allclose(out[:, 3:6], a.numpy(), atol=2e-6)
    np.testing.assert_allclose(out[:, 6], rr.numpy(), atol=2e-6)


@pytest.mark.parametrize("P,K", [(300, 5), (40, 70), (3, 1024)])
def test_trace_matches_oracle(lib, P, K):
    # few directions per point, a ragged last chunk of 32, and the distillation teacher's K
    cfg = helpers.small_cfg(levels=8)
    sc = scenegen.make_scene(cfg, 6, bias_scale=0.3)
    r = helpers.renderer_for(cfg, sc)
    rng = np.random.default_rng(7)
    feat = rng.normal(0, 0.2, (P, 16)).astype(np.float32)
    d = rng.normal(size=(P, K, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    dirs = np.zeros((P, K, 4), np.float32)
    dirs[..., :3] = d
    vis, depth = r.trace(torch.from_numpy(feat).cuda(), torch.from_numpy(dirs).cuda())
    f64 = torch.from_numpy(np.repeat(feat.astype(np.float64), K, axis=0))
    v_ref, t_ref = mlp.implicit_ray_tracer(f64, torch.from_numpy(dirs[..., :3].reshape(-1, 3).astype(np.float64)),
                                           mlp.as_layers(sc.irt), cfg.near, cfg.far)
    np.testing.assert_allclose(vis.cpu().numpy().ravel(), v_ref.numpy(), atol=3e-6)
    np.testing.assert_allclose(depth.cpu().numpy().ravel(), t_ref.numpy(), atol=3e-6)


@pytest.mark.parametrize("level", [0, 1])
def test_sample_matches_oracle(lib, level):
    cfg = helpers.small_cfg(n_dirs=24, m_dirs=5)
    r = helpers.renderer_for(cfg, scenegen.make_scene(cfg, 0))
    gb = scenegen.make_gbuffer(200, 9)
    off = 12345
    dirs = r.sample(torch.from_numpy(gb["normal"]).cuda(), level, off).cpu().numpy()
    n = torch.from_numpy(gb["normal"][:, :3].astype(np.float64))
    ids = np.arange(200, dtype=np.uint64) + np.uint64(off)
    if level == 0:
        q = ids[:, None] * np.uint64(cfg.n_dirs) + np.arange(cfg.n_dirs, dtype=np.uint64)[None, :]
        ctr = sampling.counters(q, 0, cfg.m_dirs)
    else:
        ctr = sampling.counters(ids[:, None], 1 + np.arange(cfg.m_dirs, dtype=np.uint64)[None, :], cfg.m_dirs)
    u1, u2 = sampling.uniforms(cfg.dir_seed, ctr)
    ref = sampling.cosine_direction(n[:, None, :], u1, u2).numpy()
    np.testing.assert_allclose(dirs[..., :3], ref, atol=2e-6)


@pytest.mark.parametrize("level", [0, 1])
def test_shade_matches_oracle(lib, level):
    cfg = helpers.small_cfg(n_dirs=40, m_dirs=6)
    sc = scenegen.make_scene(cfg, 2)
    r = helpers.renderer_for(cfg, sc)
    P = 257
    gb = scenegen.make_gbuffer(P, 11)
    K = cfg.n_dirs if level == 0 else cfg.m_dirs
    rng = np.random.default_rng(12)
    vis = rng.uniform(0, 1, (P, K)).astype(np.float32)
    lin = np.zeros((P, K, 4), np.float32)
    lin[..., :3] = rng.uniform(0, 2, (P, K, 3))
    pts = helpers.to_cuda(gb)
    out = r.shade(pts, level, torch.from_numpy(vis).cuda(),
                  torch.from_numpy(lin).cuda() if level == 0 else None, index_offset=77).cpu().numpy()
    n = torch.from_numpy(gb["normal"][:, :3].astype(np.float64))
    ids = np.arange(P, dtype=np.uint64) + np.uint64(77)
    if level == 0:
        ctr = sampling.counters(ids[:, None] * np.uint64(cfg.n_dirs) + np.arange(K, dtype=np.uint64)[None, :], 0,
                                cfg.m_dirs)
    else:
        ctr = sampling.counters(ids[:, None], 1 + np.arange(K, dtype=np.uint64)[None, :], cfg.m_dirs)
    u1, u2 = sampling.uniforms(cfg.dir_seed, ctr)
    w = sampling.cosine_direction(n[:, None, :], u1, u2)
    env = torch.from_numpy(sc.env.astype(np.float64))
    v = torch.from_numpy(vis.astype(np.float64))[..., None]
    li = v * shading.env_lookup(env, w)
    if level == 0:
        li = li + (1 - v) * torch.from_numpy(lin[..., :3].astype(np.float64))
    ar = torch.from_numpy(gb["albedo_rough"].astype(np.float64))
    fr = shading.brdf(ar[:, None, :3], ar[:, None, 3], n[:, None, :], w,
                      torch.from_numpy(gb["view"][:, None, :3].astype(np.float64)), cfg.f0)
    ref = shading.mc_sum(li * fr, K).numpy()
    assert helpers.rel_err(out[:, :3], ref) <= 1e-4
    assert np.all(out[:, 3] == 0)
