"""rt_render_frame_static: the FP32 render for callers that cannot allocate device memory.

Such callers (hosts whose memory manager owns all device allocations, or
frame loops with a fixed device-memory budget) get the fused kernel with its
packed-weight workspace in a static device array instead of a context.  The
two entry points run the same kernel on the same packed weights, so their
frames must be bit-identical.  This file is collected last so that a failure
here leaves every other test run; it passes alone in a fresh process (the
first call does the per-device set-up) and after the other tests.
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


def _model(sc):
    return (torch.from_numpy(sc.table).cuda(), torch.from_numpy(sc.brdf_blob).cuda(),
            torch.from_numpy(sc.irt_blob).cuda(), torch.from_numpy(np.ascontiguousarray(sc.env)).cuda())


def _static_call(lib, cfg_c, model, dgb, out, offset=0):
    g = lib.gbuffer(dgb)
    return lib.LIB.rt_render_frame_static(ctypes.byref(cfg_c), *(ctypes.c_void_p(t.data_ptr()) for t in model),
                                          ctypes.byref(g), dgb["pos"].shape[0], offset,
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _static_render(lib, cfg_c, sc, dgb, offset=0):
    model = _model(sc)
    out = torch.full((dgb["pos"].shape[0], 4), float("nan"), device="cuda")
    st = _static_call(lib, cfg_c, model, dgb, out, offset)
    assert st == lib.RT_OK, lib.status_str(st)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("mode", [{}, {"visibility": 1}])
def test_static_entry_equals_context_entry_twice(lib, mode):
    cfg = helpers.small_cfg(n_dirs=64, m_dirs=8, levels=8, log2_T=14)
    cfg_c = lib.make_config(cfg, **mode)
    dgb = helpers.to_cuda(scenegen.make_gbuffer(97, 4))
    # two calls in a row with different models and pixel offsets: the shared
    # array must follow each call, and the RNG must follow the offset
    for seed, offset in ((0, 0), (1, 12345)):
        sc = scenegen.make_scene(cfg, seed, bias_scale=0.1)
        ref = helpers.renderer_for(cfg, sc, **mode).render_frame(dgb, pixel_offset=offset).cpu().numpy()
        got = _static_render(lib, cfg_c, sc, dgb, offset)
        assert np.isfinite(got).all()
        np.testing.assert_array_equal(got, ref)
        assert np.all(got[:, 3] == 0)


def test_static_entry_allocates_no_device_memory(lib):
    cfg = helpers.small_cfg(n_dirs=32, m_dirs=8, levels=8, log2_T=14)
    cfg_c = lib.make_config(cfg)
    sc = scenegen.make_scene(cfg, 2)
    model = _model(sc)
    dgb = helpers.to_cuda(scenegen.make_gbuffer(256, 6))
    out = torch.empty(256, 4, device="cuda")
    assert _static_call(lib, cfg_c, model, dgb, out) == lib.RT_OK   # set-up and module load happen here
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        assert _static_call(lib, cfg_c, model, dgb, out) == lib.RT_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_reserved() == reserved0
    assert torch.equal(out, first)


def test_static_entry_rejects_what_it_cannot_hold(lib):
    cfg = helpers.small_cfg()
    null = ctypes.c_void_p()

    def call(c):
        return lib.LIB.rt_render_frame_static(ctypes.byref(c), null, null, null, null, None, 1, 0, null, null)
    assert call(lib.make_config(cfg, precision=lib.RT_BF16)) == lib.RT_ERR_UNSUPPORTED
    # MIS draws from a bound map's texel CDFs, which only a context holds
    assert call(lib.make_config(cfg, sampling=lib.RT_SAMPLE_MIS)) == lib.RT_ERR_UNSUPPORTED
    assert call(lib.make_config(cfg, levels=17)) == lib.RT_ERR_INVALID_ARG
    ok = lib.make_config(cfg)
    assert lib.LIB.rt_render_frame_static(ctypes.byref(ok), null, null, null, null, None, 0, 0, null, null) == lib.RT_OK
