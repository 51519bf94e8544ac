"""rt_render_frame_static: the FP32 render for callers that cannot allocate device memory.

Such callers (hosts whose memory manager owns all device allocations, or
frame loops with a fixed device-memory budget) get the fused kernel with its
packed-weight workspace in a static device array instead of a context.  This
file is collected last so that a failure here leaves every other test run;
it passes alone in a fresh process (the first call does the per-device set-up)
and after the other tests.
"""
import ctypes

import numpy as np
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


def _static_render(lib, cfg_c, sc, dgb):
    keep = (torch.from_numpy(sc.table).cuda(), torch.from_numpy(sc.brdf_blob).cuda(),
            torch.from_numpy(sc.irt_blob).cuda(), torch.from_numpy(np.ascontiguousarray(sc.env)).cuda())
    out = torch.full((dgb["pos"].shape[0], 4), float("nan"), device="cuda")
    g = lib.gbuffer(dgb)
    st = lib.LIB.rt_render_frame_static(ctypes.byref(cfg_c), *(ctypes.c_void_p(t.data_ptr()) for t in keep),
                                        ctypes.byref(g), dgb["pos"].shape[0], 0, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == lib.RT_OK, lib.status_str(st)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_static_entry_matches_context_entry_twice(lib):
    cfg = helpers.small_cfg(n_dirs=64, m_dirs=8, levels=8, log2_T=14)
    cfg_c = lib.make_config(cfg)
    dgb = helpers.to_cuda(scenegen.make_gbuffer(97, 4))
    # two calls in a row with different models: the shared array must follow each call
    for seed in (0, 1):
        sc = scenegen.make_scene(cfg, seed, bias_scale=0.1)
        ref = helpers.renderer_for(cfg, sc).render_frame(dgb).cpu().numpy()
        got = _static_render(lib, cfg_c, sc, dgb)
        assert np.isfinite(got).all()
        assert helpers.rel_err(got[:, :3], ref[:, :3]) <= helpers.FP32_PIXEL_TOL
        assert np.all(got[:, 3] == 0)


def test_static_entry_rejects_what_it_cannot_hold(lib):
    cfg = helpers.small_cfg()
    bf = lib.make_config(cfg, precision=lib.RT_BF16)
    null = ctypes.c_void_p()
    assert lib.LIB.rt_render_frame_static(ctypes.byref(bf), null, null, null, null, None, 1, 0, null, null) == \
        lib.RT_ERR_UNSUPPORTED
    bad = lib.make_config(cfg, levels=17)
    assert lib.LIB.rt_render_frame_static(ctypes.byref(bad), null, null, null, null, None, 1, 0, null, null) == \
        lib.RT_ERR_INVALID_ARG
    ok = lib.make_config(cfg)
    assert lib.LIB.rt_render_frame_static(ctypes.byref(ok), null, null, null, null, None, 0, 0, null, null) == lib.RT_OK
