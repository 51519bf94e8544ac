"""Seeded synthetic inputs for the hash-grid secondary-ray renderer.

This module only draws random numbers.  It holds none of the renderer's
arithmetic (no encoding, no MLP, no sampling, no shading), so the FP64
oracle under ``oracle/`` and the CUDA path can both consume what it makes
without sharing any of the method's code.

Every scene stands in for one of the paper's 800x800 object renders
(Sec. 4.1): the paper's datasets and trained weights are not available,
so the primary G-buffer that its CNN renderer G would produce (Sec. 3.2,
"Direct Illumination Renderer") is drawn at random, as are the hash
tables, the MLP weights and the environment map.

Distributions:
  pos            U[-1, 1]^3
  normal, view   N(0, I3), normalised (uniform on the sphere)
  albedo         U(0, 1)^3
  roughness      U(0.09, 1)   (the range the paper's remap allows, Sec. 3.3)
  table          U(-1e-4, 1e-4) * 1e3 = U(-0.1, 0.1)
  MLP weights    Xavier-uniform with the true fan-in/fan-out; biases zero
                 unless ``bias_scale`` > 0
  env map        exp(N(0, 1)) per texel and channel (lognormal RGB)
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Tuple

import numpy as np

HIDDEN = 64          # width of both MLPs (Sec. 4.1: "hidden dimensions set to 64")
PE_DIM = 27          # [w, sin(2^k pi w), cos(2^k pi w)], k = 0..3
BRDF_OUT = 7         # [n(3), a(3), r(1)]
IRT_OUT = 2          # [visibility logit, depth logit]


@dataclasses.dataclass(frozen=True)
class SceneConfig:
    """Sizes and constants of one workload."""
    name: str
    width: int
    height: int
    n_dirs: int            # N: secondary directions per primary point
    m_dirs: int = 8        # M: directions per secondary point (Sec. 4 supplementary, rendering details)
    levels: int = 16       # L
    feat_dim: int = 2      # F
    log2_T: int = 19       # T = 2^log2_T entries per level
    base_res: int = 16
    max_res: int = 2048
    env_h: int = 64
    env_w: int = 128
    precision: str = "fp32"   # "fp32" or "bf16" (FP16 table, BF16 MLPs)
    near: float = 0.05
    far: float = 1.5
    f0: float = 0.04
    dir_seed: int = 0x5EED

    @property
    def n_pixels(self) -> int:
        return self.width * self.height

    @property
    def samples(self) -> int:
        """Secondary samples per frame: P * N."""
        return self.n_pixels * self.n_dirs


# The five workloads: a tiny FP32 frame, the 800x800 FP32 frame, its BF16
# variant, the differentiation batch and the batched 1080p serving frame.
CONFIGS: Dict[str, SceneConfig] = {
    "tiny64": SceneConfig("tiny64", 64, 64, 32, levels=8, log2_T=14, base_res=16,
                          max_res=256, env_h=16, env_w=32),
    "frame800": SceneConfig("frame800", 800, 800, 128),
    "frame800_bf16": SceneConfig("frame800_bf16", 800, 800, 128, precision="bf16"),
    "grad65k": SceneConfig("grad65k", 256, 256, 64),
    "serve1080": SceneConfig("serve1080", 1920, 1080, 256, log2_T=20, precision="bf16"),
}


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def _unit(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def make_gbuffer(n_pixels: int, seed: int) -> Dict[str, np.ndarray]:
    """Random primary surface points: four float32 [P, 4] planes.

    pos.xyz U[-1,1]^3; normal.xyz and view.xyz (towards the camera) unit
    vectors; albedo_rough = (albedo rgb, roughness).  The fourth lane of
    pos/normal/view is 0.
    """
    rng = _rng(seed, 1)
    pos = np.zeros((n_pixels, 4), np.float32)
    pos[:, :3] = rng.uniform(-1.0, 1.0, (n_pixels, 3))
    normal = np.zeros((n_pixels, 4), np.float32)
    normal[:, :3] = _unit(rng, n_pixels)
    view = np.zeros((n_pixels, 4), np.float32)
    view[:, :3] = _unit(rng, n_pixels)
    ar = np.zeros((n_pixels, 4), np.float32)
    ar[:, :3] = rng.uniform(0.0, 1.0, (n_pixels, 3))
    ar[:, 3] = rng.uniform(0.09, 1.0, n_pixels)
    return {"pos": pos, "normal": normal, "view": view, "albedo_rough": ar}


def make_table(levels: int, log2_T: int, feat_dim: int, seed: int) -> np.ndarray:
    """Hash tables [L][T][F], float32, U(-1e-4, 1e-4) * 1e3."""
    rng = _rng(seed, 2)
    return (rng.uniform(-1e-4, 1e-4, (levels, 1 << log2_T, feat_dim)) * 1e3).astype(np.float32)


def _xavier(rng: np.random.Generator, fan_out: int, fan_in: int) -> np.ndarray:
    bound = math.sqrt(6.0 / (fan_in + fan_out))
    return rng.uniform(-bound, bound, (fan_out, fan_in)).astype(np.float32)


def make_mlp(in_dim: int, out_dim: int, seed: int, stream: int,
             bias_scale: float = 0.0) -> List[Tuple[np.ndarray, np.ndarray]]:
    """Three linear layers in -> 64 -> 64 -> out, as (W [out][in], b [out]) pairs."""
    rng = _rng(seed, stream)
    dims = [in_dim, HIDDEN, HIDDEN, out_dim]
    layers = []
    for a, b in zip(dims[:-1], dims[1:]):
        w = _xavier(rng, b, a)
        bias = (rng.uniform(-bias_scale, bias_scale, b) if bias_scale > 0
                else np.zeros(b)).astype(np.float32)
        layers.append((w, bias))
    return layers


def make_env(h: int, w: int, seed: int) -> np.ndarray:
    """Environment map [H][W][4] float32: lognormal(0, 1) RGB, alpha 0."""
    rng = _rng(seed, 4)
    env = np.zeros((h, w, 4), np.float32)
    env[:, :, :3] = np.exp(rng.standard_normal((h, w, 3)))
    return env


def pack_mlp(layers: List[Tuple[np.ndarray, np.ndarray]]) -> np.ndarray:
    """Concatenate W1, b1, W2, b2, W3, b3 (row-major W [out][in]) into one float32 blob."""
    parts = []
    for w, b in layers:
        parts.append(np.ascontiguousarray(w, np.float32).ravel())
        parts.append(np.ascontiguousarray(b, np.float32).ravel())
    return np.concatenate(parts)


def unpack_mlp(blob: np.ndarray, in_dim: int, out_dim: int) -> List[Tuple[np.ndarray, np.ndarray]]:
    """Inverse of :func:`pack_mlp`."""
    dims = [in_dim, HIDDEN, HIDDEN, out_dim]
    out, o = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        w = blob[o:o + a * b].reshape(b, a); o += a * b
        bias = blob[o:o + b]; o += b
        out.append((w, bias))
    assert o == blob.size
    return out


def mlp_sizes(levels: int, feat_dim: int = 2) -> Tuple[int, int]:
    """Float counts of the packed BRDF-decoder and IRT blobs."""
    lf = levels * feat_dim

    def n(i, o):
        return i * HIDDEN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN * o + o
    return n(lf, BRDF_OUT), n(lf + PE_DIM, IRT_OUT)


@dataclasses.dataclass
class Scene:
    """Model parameters of one scene (tables, both MLPs, env map)."""
    cfg: SceneConfig
    table: np.ndarray                      # [L][T][F] float32
    brdf: List[Tuple[np.ndarray, np.ndarray]]
    irt: List[Tuple[np.ndarray, np.ndarray]]
    env: np.ndarray                        # [H][W][4] float32

    @property
    def brdf_blob(self) -> np.ndarray:
        return pack_mlp(self.brdf)

    @property
    def irt_blob(self) -> np.ndarray:
        return pack_mlp(self.irt)


def make_scene(cfg: SceneConfig, seed: int, env_seed: int | None = None,
               bias_scale: float = 0.0) -> Scene:
    lf = cfg.levels * cfg.feat_dim
    return Scene(
        cfg=cfg,
        table=make_table(cfg.levels, cfg.log2_T, cfg.feat_dim, seed),
        brdf=make_mlp(lf, BRDF_OUT, seed, 10, bias_scale),
        irt=make_mlp(lf + PE_DIM, IRT_OUT, seed, 11, bias_scale),
        env=make_env(cfg.env_h, cfg.env_w, seed if env_seed is None else env_seed),
    )


def subset_permutation(n: int, k: int, seed: int) -> np.ndarray:
    """First k indices of a seeded permutation of range(n)."""
    return _rng(seed, 7).permutation(n)[:k]
