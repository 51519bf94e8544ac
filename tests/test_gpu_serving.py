"""Batched lights (rt_render_frame_multi), the launch-shape autotuner and the CUDA-graph batch."""
import numpy as np
import pytest
import torch

import scenegen
from oracle import render as orender
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2409_10327_gb300 import build
    build.build()
    from paper_2409_10327_gb300 import binding
    return binding


def _envs(cfg, n, seed0=100):
    return np.stack([scenegen.make_env(cfg.env_h, cfg.env_w, seed0 + e) for e in range(n)])


def _single_light(cfg, sc, gb, env, offset=0, shape=None):
    sc2 = scenegen.Scene(cfg, sc.table, sc.brdf, sc.irt, env)
    r = helpers.renderer_for(cfg, sc2)
    if shape is not None and cfg.precision == "bf16":
        r.set_launch_shape(1, shape[1])
    return r.render_frame(gb, pixel_offset=offset).cpu().numpy()


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_multi_light_equals_single_light_renders(lib, precision):
    cfg = helpers.small_cfg(n_dirs=48, m_dirs=4, precision=precision)
    sc = scenegen.make_scene(cfg, 0, bias_scale=0.1)
    gb = helpers.to_cuda(scenegen.make_gbuffer(150, 5))
    envs = _envs(cfg, 5)
    r = helpers.renderer_for(cfg, sc)
    denv = torch.from_numpy(envs).cuda()
    shapes = [(nl, wg) for nl in (1, 2, 4, 8) for wg in (2, 3, 4)] if precision == "bf16" else [None]
    for shape in shapes:
        if shape is not None:
            r.set_launch_shape(*shape)
        out = r.render_frame_multi(gb, denv, pixel_offset=7).cpu().numpy()
        for e in range(5):
            ref = _single_light(cfg, sc, gb, envs[e], 7, shape)
            assert helpers.rel_err(out[e, :, :3], ref[:, :3]) <= 1e-5, (shape, e)
            assert np.all(out[e, :, 3] == 0)


def test_tuner_picks_a_shape_and_reproduces_it(lib):
    cfg = helpers.small_cfg(n_dirs=64, m_dirs=8, precision="bf16")
    sc = scenegen.make_scene(cfg, 1)
    gb = helpers.to_cuda(scenegen.make_gbuffer(2000, 6))
    denv = torch.from_numpy(_envs(cfg, 8)).cuda()
    r = helpers.renderer_for(cfg, sc)
    best = r.tune(gb, denv)
    nl, wg = r.launch_shape()
    assert best > 0 and nl in (1, 2, 4, 8) and wg in (2, 3, 4) and r.tile_shape() in (32, 64, 128)
    tuned = r.render_frame_multi(gb, denv).cpu().numpy()
    r.set_launch_shape(1, 2)
    ref = r.render_frame_multi(gb, denv).cpu().numpy()
    assert helpers.rel_err(tuned[..., :3], ref[..., :3]) <= 1e-5


def test_graph_batch_matches_eager(lib):
    from paper_2409_10327_gb300 import serve
    cfg = helpers.small_cfg(n_dirs=32, m_dirs=8, precision="bf16")
    sc = scenegen.make_scene(cfg, 2)
    r = helpers.renderer_for(cfg, sc)
    gbs = [helpers.to_cuda(scenegen.make_gbuffer(300, 10 + v)) for v in range(3)]
    srv = serve.BatchedServer(r, gbs, torch.from_numpy(_envs(cfg, 3)).cuda())
    eager = srv.render_eager().clone()
    srv.capture()
    srv.out.zero_()
    got = srv.replay()
    torch.cuda.synchronize()
    assert torch.equal(got, eager)
    lat = srv.view_latencies_ms()
    assert len(lat) == 3 and all(x > 0 for x in lat)


def test_multi_light_bf16_against_oracle(lib):
    cfg = scenegen.CONFIGS["tiny64"]
    cfg = type(cfg)(**{**cfg.__dict__, "precision": "bf16"})
    sc, gb = helpers.scene_arrays(cfg, 0)
    envs = _envs(cfg, 3)
    r = helpers.renderer_for(cfg, sc)
    out = r.render_frame_multi(helpers.to_cuda(gb), torch.from_numpy(envs).cuda()).cpu().numpy()
    # every light on a seeded quarter of the frame (the whole single-light frame is checked in
    # test_gpu_render_bf16.py; multi- and single-light renders are compared in full above)
    rows = np.sort(scenegen.subset_permutation(cfg.n_pixels, cfg.n_pixels // 4, seed=2))
    for e in range(3):
        prm = orender.Params.from_arrays(sc.table, sc.brdf, sc.irt, envs[e])
        opt = helpers.oracle_options(cfg)
        ref = orender.render(gb, prm, opt, rows=rows)
        sens = orender.float32_sensitivity(gb, prm, opt, rows=rows, rel=helpers.BF16_JITTER,
                                           draws=helpers.BF16_SENS_DRAWS, mlp=True)
        ok, stats = helpers.bf16_parity(out[e, rows, :3], ref, sens)
        assert ok and stats["psnr_db"] >= helpers.BF16_PSNR_MIN, (e, stats)


def test_serve1080_full_size_multi_light_sampled(lib):
    # the 1920x1080, N=256, M=8, L=16, T=2^20 serving workload: one view, 8 env maps in one call,
    # in the launch shape the tuner picks; sampled pixels of the first and last light
    cfg = scenegen.CONFIGS["serve1080"]
    sc = scenegen.make_scene(cfg, 0)
    gb = scenegen.make_gbuffer(cfg.n_pixels, 0)
    envs = _envs(cfg, 8)
    r = helpers.renderer_for(cfg, sc)
    dgb = helpers.to_cuda(gb)
    denv = torch.from_numpy(envs).cuda()
    r.tune({k: v[:cfg.n_pixels // 8] for k, v in dgb.items()}, denv)   # as the serving bench: the first eighth
    out = r.render_frame_multi(dgb, denv).cpu().numpy()
    assert np.isfinite(out).all() and np.all(out[..., 3] == 0)
    rows = scenegen.subset_permutation(cfg.n_pixels, 48, seed=4)
    for e in (0, 7):
        prm = orender.Params.from_arrays(sc.table, sc.brdf, sc.irt, envs[e])
        opt = helpers.oracle_options(cfg)
        ref = orender.render(gb, prm, opt, rows=rows)
        sens = orender.float32_sensitivity(gb, prm, opt, rows=rows, rel=helpers.BF16_JITTER, draws=helpers.BF16_SENS_DRAWS, mlp=True)
        ok, stats = helpers.bf16_parity(out[e, rows, :3], ref, sens)
        assert ok, (e, r.launch_shape(), stats)


@pytest.mark.parametrize("n_dirs,P", [(64, 37), (128, 150), (256, 21), (48, 40)])
def test_tile_shapes_give_the_same_bits(lib, n_dirs, P):
    # 32 / 64 directions per tile (128 / d pixels per tile, the direction chunks of a pixel group walked
    # in order) against tiles of 128 consecutive samples; 48 directions: no chunked shape applies
    cfg = helpers.small_cfg(n_dirs=n_dirs, m_dirs=4, precision="bf16")
    sc = scenegen.make_scene(cfg, 3, bias_scale=0.1)
    gb = helpers.to_cuda(scenegen.make_gbuffer(P, 8))
    denv = torch.from_numpy(_envs(cfg, 4)).cuda()
    r = helpers.renderer_for(cfg, sc)
    assert r.tile_shape() == 128
    for nl, wg in ((1, 4), (4, 2)):
        r.set_launch_shape(nl, wg)
        outs = {}
        for d in (128, 64, 32):
            r.set_tile_shape(d)
            outs[d] = (r.render_frame(gb, pixel_offset=5).cpu().numpy(),
                       r.render_frame_multi(gb, denv, pixel_offset=5).cpu().numpy())
        for d in (64, 32):
            np.testing.assert_array_equal(outs[d][0], outs[128][0])
            np.testing.assert_array_equal(outs[d][1], outs[128][1])
    assert r.check() == 0
    for bad in (0, 16, 96, 256):
        with pytest.raises(lib.RtError) as e:
            r.set_tile_shape(bad)
        assert e.value.status == lib.RT_ERR_INVALID_ARG
