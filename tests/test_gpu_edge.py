"""Empty inputs through every entry point and mode: each call succeeds, launches nothing that
writes, and leaves its outputs untouched."""
import dataclasses

import pytest
import torch

import scenegen
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2409_10327_gb300 import build
    build.build()
    from paper_2409_10327_gb300 import binding
    return binding


def _empty_gb():
    return {k: torch.zeros(0, 4, device="cuda") for k in ("pos", "normal", "view", "albedo_rough")}


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("modes", [{}, {"visibility": 1}, {"sampling": 1}, {"visibility": 1, "sampling": 1}])
def test_empty_frame_every_mode(lib, precision, modes):
    cfg = helpers.small_cfg(precision=precision)
    sc, _ = helpers.scene_arrays(cfg, 0, n_pixels=4)
    r = helpers.renderer_for(cfg, sc, **modes)
    out = r.render_frame(_empty_gb())
    assert out.shape == (0, 4)
    if precision == "bf16":
        envs = torch.from_numpy(scenegen.make_env(cfg.env_h, cfg.env_w, 3)).cuda()[None].repeat(3, 1, 1, 1)
        assert r.render_frame_multi(_empty_gb(), envs).shape == (3, 0, 4)
    torch.cuda.synchronize()
    assert r.check() == 0


def test_empty_backward_and_distillation(lib):
    cfg = helpers.small_cfg()
    sc, _ = helpers.scene_arrays(cfg, 0, n_pixels=4)
    r = helpers.renderer_for(cfg, sc)
    g = [torch.zeros(n, device="cuda") for n in (sc.table.size, sc.brdf_blob.size, sc.irt_blob.size)]
    r.backward(_empty_gb(), torch.zeros(0, 4, device="cuda"), *g)
    dirs = r.distill_dirs(0, 16)
    assert dirs.shape == (0, 16, 4)
    loss = torch.zeros(3, device="cuda")
    z = torch.zeros(0, device="cuda")
    r.distill_backward(torch.zeros(0, 4, device="cuda"), torch.zeros(0, 4, device="cuda"), dirs,
                       torch.zeros(0, 8, device="cuda"), z, z, loss, *g)
    torch.cuda.synchronize()
    assert all(float(t.abs().sum()) == 0.0 for t in g + [loss])
    p = torch.zeros(0, device="cuda")
    lib.adam_step(p, p, p, p, 1)


def test_denoise_rejects_an_empty_image(lib):
    x = torch.zeros(4, 4, device="cuda")
    with pytest.raises(lib.RtError) as e:
        lib.denoise(x, torch.zeros(4, device="cuda"), x, 0, 4)
    assert e.value.status == lib.RT_ERR_INVALID_ARG


def test_largest_level_count_and_table(lib):
    # L = 16 levels (the most the kernels hold) with T = 2^22 entries per level, in both precisions,
    # against the oracle on a few pixels
    import numpy as np
    from oracle import render as orender
    for precision in ("fp32", "bf16"):
        cfg = dataclasses.replace(helpers.small_cfg(precision=precision, n_dirs=32, m_dirs=4), levels=16,
                                  log2_T=22, max_res=4096)
        sc, gb = helpers.scene_arrays(cfg, 5, bias=0.1, n_pixels=24)
        r = helpers.renderer_for(cfg, sc)
        out = r.render_frame(helpers.to_cuda(gb)).cpu().numpy()[:, :3]
        prm = helpers.oracle_params(sc)
        opt = helpers.oracle_options(cfg)
        ref = orender.render(gb, prm, opt)
        if precision == "fp32":
            sens = orender.float32_sensitivity(gb, prm, opt, draws=4)
            ok, stats = helpers.fp32_parity(out, ref, sens)
        else:
            sens = orender.float32_sensitivity(gb, prm, opt, rel=helpers.BF16_JITTER, draws=helpers.BF16_SENS_DRAWS, mlp=True)
            ok, stats = helpers.bf16_parity(out, ref, sens)
        assert ok and np.isfinite(out).all(), (precision, stats)
