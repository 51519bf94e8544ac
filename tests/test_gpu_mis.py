"""MIS primary directions (light + GGX visible normals, balance heuristic; Sec. 4.1) against the oracle."""
import dataclasses

import numpy as np
import pytest
import torch

import scenegen
from oracle import render as orender
from tests import helpers

pytestmark = pytest.mark.gpu

MIS = 1   # RT_SAMPLE_MIS


@pytest.fixture(scope="module")
def lib():
    from paper_2409_10327_gb300 import build
    build.build()
    from paper_2409_10327_gb300 import binding
    return binding


def _render(cfg, sc, gb, offset=0, **ov):
    r = helpers.renderer_for(cfg, sc, **ov)
    out = r.render_frame(helpers.to_cuda(gb), pixel_offset=offset)
    torch.cuda.synchronize()
    assert r.check() == 0
    return out.cpu().numpy()


def _bf16(cfg):
    return dataclasses.replace(cfg, precision="bf16")


@pytest.mark.parametrize("mode", [{}, {"lambert": True}])
def test_fp32_mis_frame_matches_oracle(lib, mode):
    cfg = scenegen.CONFIGS["tiny64"]
    sc, gb = helpers.scene_arrays(cfg, 0, bias=0.1)
    out = _render(cfg, sc, gb, sampling=MIS, **({"brdf_mode": 1} if mode else {}))
    prm = helpers.oracle_params(sc)
    opt = helpers.oracle_options(cfg, sampling="mis", **mode)
    ref, allow = orender.render(gb, prm, dataclasses.replace(opt, mis_margin=helpers.MIS_MARGIN))
    sens = orender.float32_sensitivity(gb, prm, opt, draws=4)
    ok, stats = helpers.fp32_parity(out[:, :3], ref, sens, extra=allow)
    assert ok, stats


def test_fp32_mis_peaked_env_matches_oracle(lib):
    # a map with one texel 1e4 times brighter and a band of near-black rows: the texel CDFs have
    # long plateaus and one large jump, so the cutpoint-guided inversion meets its edge cases
    cfg = scenegen.CONFIGS["tiny64"]
    env = scenegen.make_env(cfg.env_h, cfg.env_w, 7).copy()
    env[3, 5, :3] *= 1e4
    env[8:12, :, :3] *= 1e-6
    sc, gb = helpers.scene_arrays(cfg, 1, bias=0.1, n_pixels=600, env=env)
    out = _render(cfg, sc, gb, sampling=MIS)
    prm = helpers.oracle_params(sc)
    opt = helpers.oracle_options(cfg, sampling="mis")
    ref, allow = orender.render(gb, prm, dataclasses.replace(opt, mis_margin=helpers.MIS_MARGIN))
    sens = orender.float32_sensitivity(gb, prm, opt, draws=4)
    ok, stats = helpers.fp32_parity(out[:, :3], ref, sens, extra=allow)
    assert ok, stats


def _bf16_check(cfg, sc, gb, out, offset=0, rows=None, psnr=True, hard=False):
    prm = helpers.oracle_params(sc)
    kw = dict(sampling="mis")
    if hard:
        kw.update(hard_vis=True, decision_arith="bf16")
    opt = helpers.oracle_options(cfg, **kw)
    margins = dict(mis_margin=helpers.MIS_MARGIN, flip_margin=helpers.HARD_MARGIN_BF16 if hard else 0.0)
    ref, extra = orender.render(gb, prm, dataclasses.replace(opt, **margins), pixel_offset=offset, rows=rows)
    sens = orender.float32_sensitivity(gb, prm, opt, pixel_offset=offset, rows=rows, rel=helpers.BF16_JITTER,
                                       draws=helpers.BF16_SENS_DRAWS, mlp=True)
    got = out[:, :3] if rows is None else out[rows, :3]
    ok, stats = helpers.bf16_parity(got, ref, sens, extra=extra)
    assert ok, stats
    if psnr:
        assert stats["psnr_db"] >= helpers.BF16_PSNR_MIN, stats
    return stats


@pytest.mark.parametrize("hard", [False, True])
def test_bf16_mis_frame_matches_oracle(lib, hard):
    cfg = _bf16(scenegen.CONFIGS["tiny64"])
    sc, gb = helpers.scene_arrays(cfg, 0, bias=0.1)
    out = _render(cfg, sc, gb, sampling=MIS, **({"visibility": 1} if hard else {}))
    _bf16_check(cfg, sc, gb, out, hard=hard)


@pytest.mark.parametrize("n_dirs,m_dirs,P", [(33, 4, 40), (1, 2, 64), (2, 8, 50), (130, 3, 5)])
def test_mis_ragged_shapes(lib, n_dirs, m_dirs, P):
    # odd N (n_L = n_G + 1), N = 1 (light draws only), N = 2, pixels spanning tiles
    for precision in ("fp32", "bf16"):
        if precision == "bf16" and n_dirs < 4:
            continue   # the BF16 path needs N >= 4
        cfg = helpers.small_cfg(n_dirs=n_dirs, m_dirs=m_dirs, precision=precision)
        sc, gb = helpers.scene_arrays(cfg, 3, bias=0.2, n_pixels=P)
        out = _render(cfg, sc, gb, offset=500, sampling=MIS)
        prm = helpers.oracle_params(sc)
        opt = helpers.oracle_options(cfg, sampling="mis")
        ref, allow = orender.render(gb, prm, dataclasses.replace(opt, mis_margin=helpers.MIS_MARGIN),
                                    pixel_offset=500)
        if precision == "fp32":
            sens = orender.float32_sensitivity(gb, prm, opt, pixel_offset=500, draws=4)
            ok, stats = helpers.fp32_parity(out[:, :3], ref, sens, extra=allow)
            assert ok, stats
        else:
            _bf16_check(cfg, sc, gb, out, offset=500, psnr=False)


def test_mis_multi_light_first_light_equals_single_render(lib):
    # every light is sampled with the bound map's distribution; light 0 is the bound map itself
    cfg = helpers.small_cfg(n_dirs=48, m_dirs=4, precision="bf16")
    sc, gb = helpers.scene_arrays(cfg, 0, bias=0.1, n_pixels=120)
    envs = np.stack([sc.env] + [scenegen.make_env(cfg.env_h, cfg.env_w, 100 + e) for e in range(3)])
    r = helpers.renderer_for(cfg, sc, sampling=MIS)
    dgb = helpers.to_cuda(gb)
    for nl in (1, 4):
        r.set_launch_shape(nl, 4)
        multi = r.render_frame_multi(dgb, torch.from_numpy(envs).cuda()).cpu().numpy()
        one = r.render_frame(dgb).cpu().numpy()
        np.testing.assert_allclose(multi[0], one, rtol=1e-5, atol=1e-7 * np.abs(one).max())
        assert np.isfinite(multi).all()


def test_mis_unsupported_entry_points(lib):
    cfg = scenegen.CONFIGS["tiny64"]
    sc, gb = helpers.scene_arrays(cfg, 0, n_pixels=16)
    r = helpers.renderer_for(cfg, sc, sampling=MIS)
    dgb = helpers.to_cuda(gb)
    with pytest.raises(lib.RtError) as e:
        r.sample(dgb["normal"], 0)
    assert e.value.status == lib.RT_ERR_UNSUPPORTED
    r.sample(dgb["normal"], 1)   # the secondary sampler is unchanged
    torch.cuda.synchronize()


def test_bf16_mis_full_size_frame_sampled(lib):
    # the 800x800, N=128, M=8, L=16, T=2^19 BF16 workload with MIS primary directions, sampled pixels
    cfg = scenegen.CONFIGS["frame800_bf16"]
    sc, gb = helpers.scene_arrays(cfg, 0)
    out = _render(cfg, sc, gb, sampling=MIS)
    assert np.isfinite(out).all() and np.all(out[:, 3] == 0)
    rows = scenegen.subset_permutation(cfg.n_pixels, 192, seed=2)
    _bf16_check(cfg, sc, gb, out, rows=rows, psnr=False)


def test_fp32_mis_full_size_frame_sampled(lib):
    cfg = scenegen.CONFIGS["frame800"]
    sc, gb = helpers.scene_arrays(cfg, 0)
    out = _render(cfg, sc, gb, sampling=MIS)
    assert np.isfinite(out).all()
    rows = scenegen.subset_permutation(cfg.n_pixels, 96, seed=3)
    prm = helpers.oracle_params(sc)
    opt = helpers.oracle_options(cfg, sampling="mis")
    ref, allow = orender.render(gb, prm, dataclasses.replace(opt, mis_margin=helpers.MIS_MARGIN), rows=rows)
    sens = orender.float32_sensitivity(gb, prm, opt, rows=rows, draws=4)
    ok, stats = helpers.fp32_parity(out[rows, :3], ref, sens, extra=allow)
    assert ok, stats
