"""The library's failure paths, driven without faulting or hanging the GPU.

* A bounded device-side wait that runs out (the mbarrier wait of the tensor-
  core kernels, on a barrier nothing arrives on) records a timeout in the
  context's status word, which rt_check reports as RT_ERR_TIMEOUT; the
  context keeps rendering afterwards.
* A device allocation of rt_create that fails (injected on the host) gives
  RT_ERR_OOM, leaves no context behind and leaks nothing.
"""
import ctypes
import time

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


def test_bounded_wait_runs_out_and_reports_timeout(lib):
    cfg = helpers.small_cfg(n_dirs=32, precision="bf16")
    sc, gb = helpers.scene_arrays(cfg, 0, n_pixels=64)
    r = helpers.renderer_for(cfg, sc)
    assert r.check() == 0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    assert lib.LIB.rt_selftest_wait(r.ctx, 50_000_000, stream) == lib.RT_OK     # 50 ms limit
    word = ctypes.c_uint32(0)
    st = lib.LIB.rt_check(r.ctx, ctypes.byref(word), stream)                    # synchronises
    waited = time.perf_counter() - t0
    assert st == lib.RT_ERR_TIMEOUT, lib.status_str(st)
    assert word.value == (1 << 28) | 0xF
    assert 0.04 <= waited < 5.0, waited
    # the status word was cleared and the context still renders
    assert r.check() == 0
    out = r.render_frame(helpers.to_cuda(gb))
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    assert r.check() == 0
    assert lib.LIB.rt_selftest_wait(None, 1, stream) == lib.RT_ERR_INVALID_ARG


def test_failed_workspace_allocation_reports_oom_and_leaks_nothing(lib):
    cfg = helpers.small_cfg()
    c = lib.make_config(cfg)
    torch.cuda.synchronize()
    h = ctypes.c_void_p()
    assert lib.LIB.rt_create(ctypes.byref(c), ctypes.byref(h)) == lib.RT_OK   # module load, kernel attributes
    assert lib.LIB.rt_destroy(h) == lib.RT_OK
    free0, _ = torch.cuda.mem_get_info()
    for n in (1, 2, 3, 4):           # each of rt_create's four workspace allocations in turn
        for _ in range(40):
            assert lib.LIB.rt_debug_fail_alloc(n) == lib.RT_OK
            h = ctypes.c_void_p(12345)
            assert lib.LIB.rt_create(ctypes.byref(c), ctypes.byref(h)) == lib.RT_ERR_OOM
            assert h.value is None
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # had rt_create kept what it allocated before the failing call, 40 failures at n >= 2 would hold
    # at least 40 x 61 KB; nothing may remain
    assert free1 >= free0 - (1 << 20), (free0, free1)
    # the injection fires once: the next context is created and renders
    assert lib.LIB.rt_debug_fail_alloc(0) == lib.RT_OK
    assert lib.LIB.rt_debug_fail_alloc(-1) == lib.RT_ERR_INVALID_ARG
    sc, gb = helpers.scene_arrays(cfg, 0, n_pixels=16)
    r = helpers.renderer_for(cfg, sc)
    out = r.render_frame(helpers.to_cuda(gb)).cpu().numpy()
    assert np.isfinite(out).all()
    r.close()
