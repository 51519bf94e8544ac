"""Shared test plumbing: scenes as numpy arrays and as CUDA tensors, error metrics."""
from __future__ import annotations

import dataclasses

import numpy as np

import scenegen
from oracle import render as orender


def scene_arrays(cfg: scenegen.SceneConfig, seed: int = 0, bias: float = 0.0, n_pixels: int | None = None,
                 env: np.ndarray | None = None):
    sc = scenegen.make_scene(cfg, seed, bias_scale=bias)
    if env is not None:
        sc.env = env
    gb = scenegen.make_gbuffer(cfg.n_pixels if n_pixels is None else n_pixels, seed)
    return sc, gb


def oracle_params(sc: scenegen.Scene) -> orender.Params:
    return orender.Params.from_arrays(sc.table, sc.brdf, sc.irt, sc.env)


def oracle_options(cfg, **kw) -> orender.Options:
    return orender.Options.from_config(cfg, **kw)


def rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    """max |got - ref| / max(|ref|, 1e-6 * peak) over pixels and channels."""
    peak = float(np.abs(ref).max()) if ref.size else 1.0
    den = np.maximum(np.abs(ref), 1e-6 * peak)
    return float((np.abs(got - ref) / den).max()) if ref.size else 0.0


# FP32 parity criterion.  The exact radiance is ill-conditioned at float32
# scale on rare pixels (a grazing sample under a sharp specular lobe, or a
# secondary point on the finest hash level), where one float32 rounding of x'
# or of a sampled direction moves the FP64 result itself by up to ~1e-2.
# So the 1e-4 relative bound is applied (1) frame-wise, as the relative L1
# error, widened by the frame's total response of the oracle to float32-sized
# jitter of those inputs (render.float32_sensitivity) relative to its total
# radiance, and (2) per pixel and channel, widened by 64 times that response.
# The frame-wise widening matters under MIS primary directions (Sec. 4.1):
# GGX samples concentrate in the sharp lobes where one rounding of a
# direction moves D the most, and on the 800x800 workload the oracle's total
# response is 5.4e-4 of the frame (2.1e-4 with cosine sampling).
FP32_FRAME_TOL = 1e-4
FP32_PIXEL_TOL = 1e-4
FP32_SENS_FACTOR = 64.0


def fp32_parity(got: np.ndarray, ref: np.ndarray, sens: np.ndarray, extra=None):
    """(ok, stats) for the FP32 criterion above; `extra` widens the per-pixel bound (flip allowance)."""
    err = np.abs(got - ref)
    peak = float(np.abs(ref).max())
    bound = FP32_PIXEL_TOL * np.maximum(np.abs(ref), 1e-6 * peak) + FP32_SENS_FACTOR * sens
    if extra is not None:
        bound = bound + extra * (1.0 + FP32_PIXEL_TOL)   # the allowed terms are computed at the kernel's precision
    total = max(np.abs(ref).sum(), 1e-300)
    frame = float(err.sum() / total)
    frame_bound = FP32_FRAME_TOL + float(sens.sum() / total)
    over = err > bound
    plain = err > FP32_PIXEL_TOL * np.maximum(np.abs(ref), 1e-6 * peak)
    stats = {"frame_rel_l1": frame, "frame_bound": frame_bound, "pixels_over_bound": int(over.any(-1).sum()),
             "pixels_over_plain_1e-4": int(plain.any(-1).sum()), "max_rel": rel_err(got, ref),
             "pixels": int(ref.shape[0])}
    return frame <= frame_bound and not over.any(), stats


# BF16 criterion.  The spec bar is PSNR >= 45 dB against the FP64
# oracle (peak = max of the oracle image), applied to frames shaped like the
# paper's (N >= 32, M = 8).  With bf16 weights and activations the depth t,
# and so x', carries ~2^-8 relative error, which moves the finest hash levels
# by up to a cell, and the rounded weights bias every sample the same way; on
# degenerate shapes (N = 4, M = 1) single samples dominate a pixel and the
# exact result itself moves by tens of percent under such perturbations.  So
# every BF16 comparison also bounds each pixel by 2e-2 |ref| plus 16 times
# the oracle's response to bf16-sized (unit roundoff 2^-8) perturbations of
# x', the sphere points, the MLP activations and weights, and FP16-sized ones
# of the table (render.float32_sensitivity with mlp=True).
BF16_PSNR_MIN = 45.0
BF16_PIXEL_TOL = 2e-2
BF16_SENS_FACTOR = 16.0
BF16_JITTER = 2.0 ** -8
# The response to bf16-sized perturbations is heavy-tailed on pixels dominated
# by a sharp specular lobe (alpha = r^2 down to 0.0081): a rare draw swings the
# lobe across a sample direction.  The maximum over 4 random draws missed it
# on two pixels of the 64x64 frame (0.097 against 0.76 over 16 draws, where
# 64 draws give the same), so the BF16 bounds take 16 draws.
BF16_SENS_DRAWS = 16

# Hard visibility decides an integer (v = 1[z0 > 0]) from floating point, so
# the oracle takes it in the kernel's arithmetic (render.Options.decision_arith).
# What is left between that emulation and a kernel is summation order and fast
# transcendentals, which move a logit by far less than these margins; the rows
# whose logit lies within the margin of 0 may still go either way, and each
# such row widens its pixel's bound by what flipping it could change
# (render.Options.flip_margin).
HARD_MARGIN_FP32 = 1e-4
HARD_MARGIN_BF16 = 4e-3

# MIS weights read the light density of the texel a direction falls in, which
# jumps at texel edges; a kernel's float32 direction can land across an edge
# from the oracle's.  Directions within this angle (radians) of an edge widen
# their pixel's bound by the weight change the neighbouring texel would give
# (render.Options.mis_margin).
MIS_MARGIN = 2e-5


def bf16_parity(got: np.ndarray, ref: np.ndarray, sens: np.ndarray, extra=None):
    """(per-pixel bound holds, stats) for the BF16 criterion above; `extra` widens the per-pixel bound."""
    err = np.abs(got - ref)
    peak = float(np.abs(ref).max())
    bound = BF16_PIXEL_TOL * np.maximum(np.abs(ref), 1e-6 * peak) + BF16_SENS_FACTOR * sens
    if extra is not None:
        bound = bound + extra * (1.0 + BF16_PIXEL_TOL)   # the allowed terms are computed at the kernel's precision
    stats = {"psnr_db": psnr(got, ref), "max_abs": float(err.max()),
             "frame_rel_l1": float(err.sum() / max(np.abs(ref).sum(), 1e-300)),
             "median_rel": float(np.median(err / np.maximum(np.abs(ref), 1e-6 * peak))),
             "pixels_over_bound": int((err > bound).any(-1).sum()), "pixels": int(ref.shape[0])}
    return stats["pixels_over_bound"] == 0, stats


def psnr(got: np.ndarray, ref: np.ndarray) -> float:
    peak = float(np.abs(ref).max())
    mse = float(((got - ref) ** 2).mean())
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)


def small_cfg(**kw) -> scenegen.SceneConfig:
    base = scenegen.SceneConfig("t", 8, 8, 32, m_dirs=8, levels=8, log2_T=14, base_res=16, max_res=256,
                                env_h=16, env_w=32)
    return dataclasses.replace(base, **kw)


# ---- device side (imported lazily so CPU-only tests never touch CUDA) ------

def to_cuda(gb: dict):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in gb.items()}


def renderer_for(cfg, sc: scenegen.Scene, **overrides):
    import torch
    from paper_2409_10327_gb300 import binding
    r = binding.Renderer(binding.make_config(cfg, **overrides))
    if cfg.precision == "bf16":
        table = torch.from_numpy(sc.table).cuda().half()
    else:
        table = torch.from_numpy(sc.table).cuda()
    r.set_params(table, torch.from_numpy(sc.brdf_blob).cuda(), torch.from_numpy(sc.irt_blob).cuda(),
                 torch.from_numpy(np.ascontiguousarray(sc.env)).cuda())
    return r
