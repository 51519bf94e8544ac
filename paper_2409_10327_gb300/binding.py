"""Thin ctypes binding of ``include/rt.h`` (argument marshalling only).

Every function here forwards to the C ABI of ``librt_gb300.so`` with the same
name minus the ``rt_`` prefix where it is a method of :class:`Renderer`.
Tensors are torch CUDA tensors; their device pointers and the current CUDA
stream are passed straight through.  Nothing is computed in Python: if the
library is missing, importing this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librt_gb300.so")

RT_OK, RT_ERR_INVALID_ARG, RT_ERR_UNSUPPORTED, RT_ERR_OOM, RT_ERR_CUDA, RT_ERR_TIMEOUT, RT_ERR_BOUNDS, \
    RT_ERR_NOT_READY = range(8)
RT_FP32, RT_BF16 = 0, 1
RT_DISNEY, RT_LAMBERT = 0, 1
RT_VIS_SOFT, RT_VIS_HARD = 0, 1
RT_SAMPLE_COSINE, RT_SAMPLE_MIS = 0, 1

# Every symbol include/rt.h declares.
EXPORTS = ["rt_status_str", "rt_config_default", "rt_config_validate", "rt_level_resolution",
           "rt_level_is_dense", "rt_param_count", "rt_workspace_bytes", "rt_create", "rt_destroy",
           "rt_set_params", "rt_check", "rt_encode", "rt_decode", "rt_trace", "rt_sample", "rt_shade",
           "rt_render_frame", "rt_backward", "rt_render_frame_static", "rt_render_frame_multi", "rt_tune",
           "rt_tuned_shape", "rt_set_launch_shape", "rt_tuned_tile_shape", "rt_set_tile_shape", "rt_denoise", "rt_distill_dirs",
           "rt_distill_backward", "rt_adam_step", "rt_selftest_wait", "rt_debug_fail_alloc",
           "rt_probe_gather", "rt_probe_ffma"]


class RtConfig(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("feat_dim", ctypes.c_int32), ("log2_T", ctypes.c_int32),
                ("base_res", ctypes.c_int32), ("max_res", ctypes.c_int32), ("dense_coarse", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("n_dirs", ctypes.c_int32), ("m_dirs", ctypes.c_int32),
                ("brdf_mode", ctypes.c_int32), ("near_t", ctypes.c_float), ("far_t", ctypes.c_float),
                ("f0", ctypes.c_float), ("force_vis", ctypes.c_float), ("force_vis2", ctypes.c_float),
                ("visibility", ctypes.c_int32), ("sampling", ctypes.c_int32), ("env_h", ctypes.c_int32),
                ("env_w", ctypes.c_int32),
                ("dir_seed", ctypes.c_uint64)]


class RtGbuffer(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("normal", ctypes.c_void_p), ("view", ctypes.c_void_p),
                ("albedo_rough", ctypes.c_void_p)]


class RtError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {status_str(status)} ({status})")
        self.status = status


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2409_10327_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U32, F32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float
    cfgp = ctypes.POINTER(RtConfig)
    sig = {
        "rt_status_str": (ctypes.c_char_p, [I32]),
        "rt_config_default": (I32, [cfgp]),
        "rt_config_validate": (I32, [cfgp]),
        "rt_level_resolution": (I32, [cfgp, I32]),
        "rt_level_is_dense": (I32, [cfgp, I32]),
        "rt_param_count": (I64, [cfgp, I32]),
        "rt_workspace_bytes": (I64, [cfgp]),
        "rt_create": (I32, [cfgp, ctypes.POINTER(P)]),
        "rt_destroy": (I32, [P]),
        "rt_set_params": (I32, [P, P, P, P, P, P]),
        "rt_check": (I32, [P, ctypes.POINTER(U32), P]),
        "rt_encode": (I32, [P, P, I64, P, P, P, P]),
        "rt_decode": (I32, [P, P, I64, P, P]),
        "rt_trace": (I32, [P, P, P, I64, I32, P, P, P]),
        "rt_sample": (I32, [P, P, I64, I32, I64, P, P]),
        "rt_shade": (I32, [P, ctypes.POINTER(RtGbuffer), I64, I32, I64, P, P, P, P]),
        "rt_render_frame": (I32, [P, ctypes.POINTER(RtGbuffer), I64, I64, P, P]),
        "rt_backward": (I32, [P, ctypes.POINTER(RtGbuffer), I64, I64, P, P, P, P, P]),
        "rt_render_frame_static": (I32, [cfgp, P, P, P, P, ctypes.POINTER(RtGbuffer), I64, I64, P, P]),
        "rt_render_frame_multi": (I32, [P, ctypes.POINTER(RtGbuffer), I64, I64, P, I32, P, P]),
        "rt_tune": (I32, [P, ctypes.POINTER(RtGbuffer), I64, I64, P, I32, P, P, ctypes.POINTER(ctypes.c_float)]),
        "rt_tuned_shape": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "rt_set_launch_shape": (I32, [P, I32, I32]),
        "rt_tuned_tile_shape": (I32, [P, ctypes.POINTER(I32)]),
        "rt_set_tile_shape": (I32, [P, I32]),
        "rt_denoise": (I32, [I32, I32, P, P, P, I32, F32, F32, F32, P, P, P]),
        "rt_distill_dirs": (I32, [P, I64, I32, I64, P, P]),
        "rt_distill_backward": (I32, [P, P, P, I64, I32, P, P, P, P, P, P, P, P, P]),
        "rt_adam_step": (I32, [P, P, P, P, I64, F32, F32, F32, F32, F32, I32, P]),
        "rt_selftest_wait": (I32, [P, I64, P]),
        "rt_debug_fail_alloc": (I32, [I32]),
        "rt_probe_gather": (I32, [P, I64, I32, I32, I32, P, P]),
        "rt_probe_ffma": (I32, [I32, I32, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def status_str(status: int) -> str:
    return LIB.rt_status_str(status).decode()


def _check(fn: str, status: int) -> None:
    if status != RT_OK:
        raise RtError(fn, status)


def make_config(cfg=None, **overrides) -> RtConfig:
    """rt_config from defaults, an object with SceneConfig-like fields, and overrides."""
    c = RtConfig()
    _check("rt_config_default", LIB.rt_config_default(ctypes.byref(c)))
    if cfg is not None:
        c.levels, c.log2_T = cfg.levels, cfg.log2_T
        c.base_res, c.max_res = cfg.base_res, cfg.max_res
        c.n_dirs, c.m_dirs = cfg.n_dirs, cfg.m_dirs
        c.env_h, c.env_w = cfg.env_h, cfg.env_w
        c.near_t, c.far_t, c.f0 = cfg.near, cfg.far, cfg.f0
        c.precision = RT_BF16 if cfg.precision == "bf16" else RT_FP32
        c.dir_seed = cfg.dir_seed
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def config_validate(c: RtConfig) -> int:
    return LIB.rt_config_validate(ctypes.byref(c))


def level_resolution(c: RtConfig, level: int) -> int:
    return LIB.rt_level_resolution(ctypes.byref(c), level)


def level_is_dense(c: RtConfig, level: int) -> int:
    return LIB.rt_level_is_dense(ctypes.byref(c), level)


def param_count(c: RtConfig, which: int) -> int:
    return LIB.rt_param_count(ctypes.byref(c), which)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensors are required")
    if not t.is_contiguous():
        raise ValueError("contiguous tensors are required")
    return ctypes.c_void_p(t.data_ptr())


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def denoise(radiance: torch.Tensor, depth: torch.Tensor, normal: torch.Tensor, width: int, height: int,
            iterations: int = 5, sigma_z: float = 1.0, sigma_n: float = 128.0, sigma_l: float = 4.0,
            out: Optional[torch.Tensor] = None, work: Optional[torch.Tensor] = None) -> torch.Tensor:
    """rt_denoise: spatial SVGF of a width x height frame; returns [P, 4] (rgb, variance)."""
    P = width * height
    out = torch.empty(P, 4, device=radiance.device, dtype=torch.float32) if out is None else out
    work = torch.empty(P, 4, device=radiance.device, dtype=torch.float32) if work is None else work
    _check("rt_denoise", LIB.rt_denoise(width, height, _ptr(radiance), _ptr(depth), _ptr(normal), iterations,
                                        sigma_z, sigma_n, sigma_l, _ptr(work), _ptr(out), _stream()))
    return out


def adam_step(param: torch.Tensor, grad: torch.Tensor, m1: torch.Tensor, m2: torch.Tensor, step: int,
              lr: float = 2e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
              weight_decay: float = 0.0) -> None:
    """rt_adam_step in place on float32 device tensors of equal size."""
    _check("rt_adam_step", LIB.rt_adam_step(_ptr(param), _ptr(grad), _ptr(m1), _ptr(m2), param.numel(), lr, beta1,
                                            beta2, eps, weight_decay, step, _stream()))


def probe_gather(table: torch.Tensor, bytes_per_load: int, iters: int, blocks: int,
                 sink: Optional[torch.Tensor] = None) -> torch.Tensor:
    """rt_probe_gather over a contiguous device table (its bytes / bytes_per_load rows)."""
    rows = table.numel() * table.element_size() // bytes_per_load
    sink = torch.empty(blocks * 512, dtype=torch.int32, device=table.device) if sink is None else sink
    _check("rt_probe_gather", LIB.rt_probe_gather(_ptr(table), rows, bytes_per_load, iters, blocks, _ptr(sink),
                                                  _stream()))
    return sink


def probe_ffma(iters: int, blocks: int, sink: Optional[torch.Tensor] = None) -> torch.Tensor:
    """rt_probe_ffma; returns the sink [blocks * 512] float."""
    sink = torch.empty(blocks * 512, dtype=torch.float32, device="cuda") if sink is None else sink
    _check("rt_probe_ffma", LIB.rt_probe_ffma(iters, blocks, _ptr(sink), _stream()))
    return sink


def gbuffer(gb: Dict[str, torch.Tensor]) -> RtGbuffer:
    return RtGbuffer(_ptr(gb["pos"]), _ptr(gb["normal"]), _ptr(gb["view"]), _ptr(gb["albedo_rough"]))


class Renderer:
    """Owns one rt_ctx; each method is one C-ABI call on the current stream."""

    def __init__(self, cfg: RtConfig):
        self.cfg = cfg
        self.levels = cfg.levels
        self.lf = 2 * cfg.levels
        h = ctypes.c_void_p()
        _check("rt_create", LIB.rt_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.ctx = h
        self._keep = ()

    def close(self) -> None:
        if self.ctx:
            LIB.rt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, table: torch.Tensor, brdf_w: torch.Tensor, irt_w: torch.Tensor, env: torch.Tensor):
        self._keep = (table, brdf_w, irt_w, env)   # the library reads table and env by reference
        _check("rt_set_params", LIB.rt_set_params(self.ctx, _ptr(table), _ptr(brdf_w), _ptr(irt_w), _ptr(env),
                                                  _stream()))

    def check(self) -> int:
        w = ctypes.c_uint32(0)
        st = LIB.rt_check(self.ctx, ctypes.byref(w), _stream())
        if st not in (RT_OK, RT_ERR_TIMEOUT, RT_ERR_BOUNDS):
            _check("rt_check", st)
        return w.value

    def encode(self, pos: torch.Tensor, want_aux: bool = False):
        P = pos.shape[0]
        feat = torch.empty(P, self.lf, device=pos.device, dtype=torch.float32)
        idx = torch.empty(P, self.levels, 8, device=pos.device, dtype=torch.int32) if want_aux else None
        w = torch.empty(P, self.levels, 8, device=pos.device, dtype=torch.float32) if want_aux else None
        _check("rt_encode", LIB.rt_encode(self.ctx, _ptr(pos), P, _ptr(feat), _ptr(idx), _ptr(w), _stream()))
        return (feat, idx, w) if want_aux else feat

    def decode(self, feat: torch.Tensor) -> torch.Tensor:
        P = feat.shape[0]
        out = torch.empty(P, 8, device=feat.device, dtype=torch.float32)
        _check("rt_decode", LIB.rt_decode(self.ctx, _ptr(feat), P, _ptr(out), _stream()))
        return out

    def trace(self, feat: torch.Tensor, dirs: torch.Tensor):
        P, K = dirs.shape[0], dirs.shape[1]
        vis = torch.empty(P, K, device=feat.device, dtype=torch.float32)
        depth = torch.empty_like(vis)
        _check("rt_trace", LIB.rt_trace(self.ctx, _ptr(feat), _ptr(dirs), P, K, _ptr(vis), _ptr(depth), _stream()))
        return vis, depth

    def sample(self, normal: torch.Tensor, level: int, index_offset: int = 0) -> torch.Tensor:
        P = normal.shape[0]
        K = self.cfg.n_dirs if level == 0 else self.cfg.m_dirs
        dirs = torch.empty(P, K, 4, device=normal.device, dtype=torch.float32)
        _check("rt_sample", LIB.rt_sample(self.ctx, _ptr(normal), P, level, index_offset, _ptr(dirs), _stream()))
        return dirs

    def shade(self, pts: Dict[str, torch.Tensor], level: int, vis: torch.Tensor, lin: Optional[torch.Tensor] = None,
              index_offset: int = 0) -> torch.Tensor:
        P = pts["normal"].shape[0]
        out = torch.empty(P, 4, device=vis.device, dtype=torch.float32)
        g = RtGbuffer(None, _ptr(pts["normal"]), _ptr(pts["view"]), _ptr(pts["albedo_rough"]))
        _check("rt_shade", LIB.rt_shade(self.ctx, ctypes.byref(g), P, level, index_offset, _ptr(vis), _ptr(lin),
                                        _ptr(out), _stream()))
        return out

    def render_frame(self, gb: Dict[str, torch.Tensor], pixel_offset: int = 0,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
        P = gb["pos"].shape[0]
        if out is None:
            out = torch.empty(P, 4, device=gb["pos"].device, dtype=torch.float32)
        g = gbuffer(gb)
        _check("rt_render_frame", LIB.rt_render_frame(self.ctx, ctypes.byref(g), P, pixel_offset, _ptr(out),
                                                      _stream()))
        return out

    def render_frame_multi(self, gb: Dict[str, torch.Tensor], envs: torch.Tensor, pixel_offset: int = 0,
                           out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Radiance [E, P, 4] of the G-buffer under the E maps envs [E, H, W, 4]."""
        P, E = gb["pos"].shape[0], envs.shape[0]
        if out is None:
            out = torch.empty(E, P, 4, device=gb["pos"].device, dtype=torch.float32)
        g = gbuffer(gb)
        _check("rt_render_frame_multi", LIB.rt_render_frame_multi(self.ctx, ctypes.byref(g), P, pixel_offset,
                                                                  _ptr(envs), E, _ptr(out), _stream()))
        return out

    def tune(self, gb: Dict[str, torch.Tensor], envs: torch.Tensor, pixel_offset: int = 0) -> float:
        """rt_tune on this workload; returns the best time in ms (-1 for FP32)."""
        P, E = gb["pos"].shape[0], envs.shape[0]
        out = torch.empty(E, P, 4, device=gb["pos"].device, dtype=torch.float32)
        best = ctypes.c_float(0.0)
        g = gbuffer(gb)
        _check("rt_tune", LIB.rt_tune(self.ctx, ctypes.byref(g), P, pixel_offset, _ptr(envs), E, _ptr(out),
                                      _stream(), ctypes.byref(best)))
        return best.value

    def launch_shape(self):
        nl, wg = ctypes.c_int32(), ctypes.c_int32()
        _check("rt_tuned_shape", LIB.rt_tuned_shape(self.ctx, ctypes.byref(nl), ctypes.byref(wg)))
        return nl.value, wg.value

    def set_launch_shape(self, lights_per_launch: int, warpgroups: int) -> None:
        _check("rt_set_launch_shape", LIB.rt_set_launch_shape(self.ctx, lights_per_launch, warpgroups))

    def tile_shape(self) -> int:
        """Directions of a pixel per 128-row tile of the BF16 kernel (128: consecutive samples)."""
        d = ctypes.c_int32()
        _check("rt_tuned_tile_shape", LIB.rt_tuned_tile_shape(self.ctx, ctypes.byref(d)))
        return d.value

    def set_tile_shape(self, dirs_per_tile: int) -> None:
        _check("rt_set_tile_shape", LIB.rt_set_tile_shape(self.ctx, dirs_per_tile))

    def render_frame_host(self, gb_host: Dict[str, torch.Tensor], out_host: torch.Tensor,
                          staging: Dict[str, torch.Tensor], out_dev: torch.Tensor, pixel_offset: int = 0) -> None:
        """rt_render_frame on host (pinned) buffers: copy the G-buffer in, render, copy the radiance out.

        All three steps are queued on the current stream; `staging` and
        `out_dev` are caller-provided device buffers of matching shapes.
        """
        for k in ("pos", "normal", "view", "albedo_rough"):
            staging[k].copy_(gb_host[k], non_blocking=True)
        self.render_frame(staging, pixel_offset, out=out_dev)
        out_host.copy_(out_dev, non_blocking=True)

    def distill_dirs(self, P: int, K: int, ray_offset: int = 0) -> torch.Tensor:
        dirs = torch.empty(P, K, 4, device="cuda", dtype=torch.float32)
        _check("rt_distill_dirs", LIB.rt_distill_dirs(self.ctx, P, K, ray_offset, _ptr(dirs), _stream()))
        return dirs

    def distill_backward(self, pos: torch.Tensor, normal: torch.Tensor, dirs: torch.Tensor, brdf_t: torch.Tensor,
                         vis_t: torch.Tensor, depth_t: torch.Tensor, loss: Optional[torch.Tensor],
                         g_table: torch.Tensor, g_brdf: torch.Tensor, g_irt: torch.Tensor) -> None:
        P, K = dirs.shape[0], dirs.shape[1]
        _check("rt_distill_backward", LIB.rt_distill_backward(
            self.ctx, _ptr(pos), _ptr(normal), P, K, _ptr(dirs), _ptr(brdf_t), _ptr(vis_t), _ptr(depth_t),
            _ptr(loss), _ptr(g_table), _ptr(g_brdf), _ptr(g_irt), _stream()))

    def backward(self, gb: Dict[str, torch.Tensor], d_radiance: torch.Tensor, g_table: torch.Tensor,
                 g_brdf: torch.Tensor, g_irt: torch.Tensor, pixel_offset: int = 0) -> None:
        P = gb["pos"].shape[0]
        g = gbuffer(gb)
        _check("rt_backward", LIB.rt_backward(self.ctx, ctypes.byref(g), P, pixel_offset, _ptr(d_radiance),
                                              _ptr(g_table), _ptr(g_brdf), _ptr(g_irt), _stream()))
