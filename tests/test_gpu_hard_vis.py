"""Hard visibility (the paper's inference, Sec. 3.2 overview): only shadow directions bounce.

The BF16 kernel queues shadow rows per warpgroup and runs them in compacted
128-row tiles; the FP32 kernel takes the same decisions without compaction.
"""
import dataclasses

import numpy as np
import pytest
import torch

import scenegen
from oracle import render as orender
from tests import helpers

pytestmark = pytest.mark.gpu

HARD = 1   # RT_VIS_HARD


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
    return type(cfg)(**{**cfg.__dict__, "precision": "bf16"})


def test_fp32_hard_frame_matches_oracle(lib):
    cfg = scenegen.CONFIGS["tiny64"]
    sc, gb = helpers.scene_arrays(cfg, 0, bias=0.1)
    out = _render(cfg, sc, gb, visibility=HARD)
    prm = helpers.oracle_params(sc)
    opt = helpers.oracle_options(cfg, hard_vis=True, decision_arith="fp32")
    ref, allow = orender.render(gb, prm, dataclasses.replace(opt, flip_margin=helpers.HARD_MARGIN_FP32))
    sens = orender.float32_sensitivity(gb, prm, opt, draws=4)
    ok, stats = helpers.fp32_parity(out[:, :3], ref, sens, extra=allow)
    assert ok, stats


def _bf16_hard_check(cfg, sc, gb, out, offset=0, rows=None, psnr=True):
    prm = helpers.oracle_params(sc)
    opt = helpers.oracle_options(cfg, hard_vis=True, decision_arith="bf16")
    ref, allow = orender.render(gb, prm, dataclasses.replace(opt, flip_margin=helpers.HARD_MARGIN_BF16),
                                pixel_offset=offset, rows=rows)
    sens = orender.float32_sensitivity(gb, prm, opt, pixel_offset=offset, rows=rows, rel=helpers.BF16_JITTER,
                                       draws=helpers.BF16_SENS_DRAWS, mlp=True)
    got = out[:, :3] if rows is None else out[rows, :3]
    ok, stats = helpers.bf16_parity(got, ref, sens, extra=allow)
    stats["pixels_with_flip_allowance"] = int((allow > 0).any(-1).sum())
    assert ok, stats
    if psnr:
        assert stats["psnr_db"] >= helpers.BF16_PSNR_MIN, stats
    return stats


def test_bf16_hard_frame_matches_oracle(lib):
    cfg = _bf16(scenegen.CONFIGS["tiny64"])
    sc, gb = helpers.scene_arrays(cfg, 0, bias=0.1)
    out = _render(cfg, sc, gb, visibility=HARD)
    assert np.all(out[:, 3] == 0)
    _bf16_hard_check(cfg, sc, gb, out)


@pytest.mark.parametrize("n_dirs,m_dirs,levels,log2_T,P", [(40, 3, 5, 12, 37), (4, 1, 1, 10, 45), (96, 8, 16, 19, 19),
                                                          (256, 2, 16, 19, 3), (33, 16, 3, 9, 64)])
def test_bf16_hard_ragged_shapes(lib, n_dirs, m_dirs, levels, log2_T, P):
    # partial queue tiles, pixels spanning several primary tiles, many pixels per tile
    cfg = helpers.small_cfg(n_dirs=n_dirs, m_dirs=m_dirs, levels=levels, log2_T=log2_T,
                            max_res=256 if levels > 1 else 16, precision="bf16")
    sc, gb = helpers.scene_arrays(cfg, 3, bias=0.2, n_pixels=P)
    out = _render(cfg, sc, gb, offset=1000, visibility=HARD)
    _bf16_hard_check(cfg, sc, gb, out, offset=1000, psnr=n_dirs >= 32 and m_dirs >= 8)


@pytest.mark.parametrize("forced", [dict(force_vis=1.0), dict(force_vis=0.0, force_vis2=1.0),
                                    dict(force_vis=0.0, force_vis2=0.0)])
@pytest.mark.parametrize("n_dirs", [48, 200])
def test_bf16_hard_with_forced_visibility_equals_soft(lib, forced, n_dirs):
    # v in {0, 1} forced: the compacted queue must reproduce the soft kernel's blend exactly
    # (all rows visible: nothing queued; all rows shadow: every row queued)
    cfg = helpers.small_cfg(n_dirs=n_dirs, m_dirs=4, precision="bf16")
    sc, gb = helpers.scene_arrays(cfg, 4, bias=0.2, n_pixels=150)
    hard = _render(cfg, sc, gb, offset=7, visibility=HARD, **forced)
    soft = _render(cfg, sc, gb, offset=7, **forced)
    np.testing.assert_allclose(hard, soft, rtol=2e-5, atol=1e-6 * np.abs(soft).max())


def test_bf16_hard_multi_light_and_determinism(lib):
    cfg = helpers.small_cfg(n_dirs=48, m_dirs=4, precision="bf16")
    sc, gb = helpers.scene_arrays(cfg, 0, bias=0.1, n_pixels=150)
    envs = np.stack([scenegen.make_env(cfg.env_h, cfg.env_w, 100 + e) for e in range(5)])
    r = helpers.renderer_for(cfg, sc, visibility=HARD)
    dgb, denv = helpers.to_cuda(gb), torch.from_numpy(envs).cuda()
    for nl in (1, 2, 4, 8):
        r.set_launch_shape(nl, 4)
        out = r.render_frame_multi(dgb, denv, pixel_offset=3).cpu().numpy()
        again = r.render_frame_multi(dgb, denv, pixel_offset=3).cpu().numpy()
        np.testing.assert_array_equal(out, again)
        for e in range(5):
            sc1 = scenegen.Scene(cfg, sc.table, sc.brdf, sc.irt, envs[e])
            one = helpers.renderer_for(cfg, sc1, visibility=HARD).render_frame(dgb, pixel_offset=3).cpu().numpy()
            np.testing.assert_allclose(out[e], one, rtol=1e-5, atol=1e-7 * np.abs(one).max())


def test_bf16_hard_sharded_frame(lib):
    cfg = helpers.small_cfg(precision="bf16")
    sc, gb = helpers.scene_arrays(cfg, 5, bias=0.1, n_pixels=300)
    r = helpers.renderer_for(cfg, sc, visibility=HARD)
    dgb = helpers.to_cuda(gb)
    whole = r.render_frame(dgb).cpu().numpy()
    parts = [r.render_frame({k: v[lo:hi].contiguous() for k, v in dgb.items()}, pixel_offset=lo).cpu().numpy()
             for lo, hi in [(0, 77), (77, 78), (78, 300)]]
    np.testing.assert_allclose(np.concatenate(parts), whole, rtol=1e-5, atol=1e-7 * np.abs(whole).max())


def test_hard_backward_is_unsupported(lib):
    cfg = scenegen.CONFIGS["tiny64"]
    sc, gb = helpers.scene_arrays(cfg, 0, n_pixels=16)
    r = helpers.renderer_for(cfg, sc, visibility=HARD)
    d = torch.zeros(16, 4, device="cuda")
    g_t = torch.zeros(sc.table.size, device="cuda")
    g_b = torch.zeros(sc.brdf_blob.size, device="cuda")
    g_i = torch.zeros(sc.irt_blob.size, device="cuda")
    with pytest.raises(lib.RtError) as e:
        r.backward(helpers.to_cuda(gb), d, g_t, g_b, g_i)
    assert e.value.status == lib.RT_ERR_UNSUPPORTED


def test_bf16_hard_full_size_frame_sampled(lib):
    cfg = scenegen.CONFIGS["frame800_bf16"]
    sc, gb = helpers.scene_arrays(cfg, 0)
    out = _render(cfg, sc, gb, visibility=HARD)
    assert np.isfinite(out).all()
    rows = scenegen.subset_permutation(cfg.n_pixels, 256, seed=0)
    _bf16_hard_check(cfg, sc, gb, out, rows=rows, psnr=False)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_hard_frame_against_fp64_decisions(lib, precision):
    # The parity tests above take the decisions in the kernel's arithmetic (with a flip allowance).
    # This one reports what the decisions themselves change: the oracle's frame with FP64 decisions
    # against the same frame with decisions in the kernel's arithmetic (pixels touched by a flipped
    # decision, and the frame L1 of the difference), and the GPU frame against both.
    cfg = scenegen.CONFIGS["tiny64"] if precision == "fp32" else _bf16(scenegen.CONFIGS["tiny64"])
    sc, gb = helpers.scene_arrays(cfg, 0, bias=0.1)
    out = _render(cfg, sc, gb, visibility=HARD)[:, :3]
    prm = helpers.oracle_params(sc)
    ref64 = orender.render(gb, prm, helpers.oracle_options(cfg, hard_vis=True, decision_arith="fp64"))
    refk = orender.render(gb, prm, helpers.oracle_options(cfg, hard_vis=True, decision_arith=precision))
    ref64, refk = np.asarray(ref64), np.asarray(refk)
    norm = np.abs(ref64).sum()
    touched = np.abs(refk - ref64).max(-1) > 1e-12 * np.maximum(np.abs(ref64).max(-1), 1e-300)
    stats = {"pixels": int(ref64.shape[0]), "pixels_touched_by_flips": int(touched.sum()),
             "flip_effect_frame_l1": float(np.abs(refk - ref64).sum() / norm),
             "gpu_vs_fp64_decisions_l1": float(np.abs(out - ref64).sum() / norm),
             "gpu_vs_kernel_decisions_l1": float(np.abs(out - refk).sum() / norm)}
    print(precision, stats)
    # flips are rare and small next to the frame; the GPU frame is closer to the kernel-arithmetic
    # decisions than to the FP64 ones wherever they differ
    assert stats["pixels_touched_by_flips"] <= 0.1 * stats["pixels"], stats
    assert stats["flip_effect_frame_l1"] <= 1e-2, stats
    assert stats["gpu_vs_kernel_decisions_l1"] <= stats["gpu_vs_fp64_decisions_l1"] + 1e-9, stats
