"""The C-ABI library loads, exports every declared symbol and validates on the host (no GPU calls)."""
import ctypes
import os
import re

import pytest

import scenegen
from oracle import hashgrid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bnd():
    from paper_2409_10327_gb300 import build
    build.build()
    from paper_2409_10327_gb300 import binding
    return binding


def _declared():
    src = open(os.path.join(ROOT, "include", "rt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(bnd):
    declared = _declared()
    assert len(declared) >= 17
    lib = ctypes.CDLL(bnd.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(bnd.EXPORTS) == declared


def test_status_strings(bnd):
    assert bnd.status_str(0) == "RT_OK"
    assert bnd.status_str(1) == "RT_ERR_INVALID_ARG"
    assert bnd.status_str(99) == "RT_ERR_UNKNOWN"


@pytest.mark.parametrize("name", ["tiny64", "frame800", "serve1080"])
def test_level_ladder_matches_oracle(bnd, name):
    cfg = scenegen.CONFIGS[name]
    c = bnd.make_config(cfg)
    assert bnd.config_validate(c) == 0
    res = hashgrid.level_resolutions(cfg.levels, cfg.base_res, cfg.max_res)
    dense = hashgrid.dense_levels(res, 1 << cfg.log2_T)
    assert [bnd.level_resolution(c, l) for l in range(cfg.levels)] == res
    assert [bnd.level_is_dense(c, l) for l in range(cfg.levels)] == [int(d) for d in dense]
    assert bnd.level_resolution(c, cfg.levels) == -1


def test_param_counts_match_blob_layout(bnd):
    for name in ["tiny64", "frame800"]:
        cfg = scenegen.CONFIGS[name]
        c = bnd.make_config(cfg)
        nb, ni = scenegen.mlp_sizes(cfg.levels)
        sc = scenegen.make_scene(cfg, 0)
        assert bnd.param_count(c, 1) == nb == sc.brdf_blob.size
        assert bnd.param_count(c, 2) == ni == sc.irt_blob.size
        assert bnd.param_count(c, 0) == sc.table.size
        assert bnd.param_count(c, 3) == -1


@pytest.mark.parametrize("field,value", [("levels", 0), ("levels", 17), ("feat_dim", 4), ("log2_T", 7),
                                         ("log2_T", 25), ("base_res", 1), ("max_res", 8), ("n_dirs", 0),
                                         ("n_dirs", 5000), ("m_dirs", 0), ("precision", 2), ("brdf_mode", 3),
                                         ("far_t", 0.01), ("f0", 1.5), ("force_vis", 2.0), ("env_h", 0),
                                         ("near_t", float("nan"))])
def test_invalid_configs_rejected(bnd, field, value):
    c = bnd.make_config(scenegen.CONFIGS["frame800"])
    setattr(c, field, value)
    assert bnd.config_validate(c) == bnd.RT_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert bnd.LIB.rt_create(ctypes.byref(c), ctypes.byref(h)) == bnd.RT_ERR_INVALID_ARG
    assert not h.value


def test_null_arguments_rejected_without_a_device(bnd):
    lib = bnd.LIB
    assert lib.rt_config_validate(None) == bnd.RT_ERR_INVALID_ARG
    assert lib.rt_create(None, None) == bnd.RT_ERR_INVALID_ARG
    assert lib.rt_destroy(None) == bnd.RT_OK
    assert lib.rt_render_frame(None, None, 0, 0, None, None) == bnd.RT_ERR_INVALID_ARG
    assert lib.rt_encode(None, None, 0, None, None, None, None) == bnd.RT_ERR_INVALID_ARG
    assert lib.rt_backward(None, None, 0, 0, None, None, None, None, None) == bnd.RT_ERR_INVALID_ARG
    w = ctypes.c_uint32()
    assert lib.rt_check(None, ctypes.byref(w), None) == bnd.RT_ERR_INVALID_ARG
