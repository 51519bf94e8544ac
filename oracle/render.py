"""The whole hash-renderer path and its FP64 gradient  (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For every primary point x with normal n, view direction w_o, albedo a and
roughness r (the G-buffer that the paper's CNN renderer G would produce;
Sec. 3.2 overview), following the paper's order (Sec. 3.1, Sec. 3.2
overview):

  (a) f = H(x)
      for each of N directions w_i (cosine-weighted about n):
  (c)     v_i, t_i = I(f, w_i)
  (d)     x'_i = x + t_i w_i;  f'_i = H(x'_i)
  (b)     a'_i, r'_i, n'_i = B(f'_i)
          for each of M directions w'_ij (cosine-weighted about n'_i):
  (c)         v'_ij = I(f'_i, w'_ij)
  (e)     L'_o,i = (pi/M) sum_j v'_ij L_env(w'_ij) f_r(a'_i, r'_i, n'_i; w'_ij, -w_i)
          L(x, w_i) = v_i L_env(w_i) + (1 - v_i) L'_o,i                 (Eq. 2)
  (e) L(x, w_o) = (pi/N) sum_i L(x, w_i) f_r(a, r, n; w_i, w_o)          (Eq. 1)

Readings: the default is the soft, differentiable form of Eq. 2 in which
every direction bounces with weight (1 - v).  `hard_vis` is the paper's
inference (Sec. 3.2 overview): I's visibility is a hit test, v = 1 when
sigma(z0) > 0.5 and 0 otherwise, for v and v' alike, so only shadow
directions (v = 0) bounce and only visible secondary directions (v' = 1)
count at x'; Eq. 2 is unchanged with V in {0, 1}.  The hit test decides an
integer from floating point, so it is taken in the arithmetic of the kernel
under test (`decision_arith`: 'fp64', 'fp32' or 'bf16'; see
`_kernel_logits`); the radiance given those decisions stays float64.
`flip_margin` > 0 also returns, per pixel, what flipping the decision of
every row whose logit lies within that margin of 0 could change (the rows a
kernel may decide the other way through its own rounding).  `force_vis`
and `force_vis2` pin v or v' to a constant (used by the furnace tests);
`lambert` drops the specular lobe.  There is no third bounce: the secondary
sum keeps only the environment light that reaches x' (v'), as in the
paper's "collect only visible rays".

Gradient (distillation pattern): the loss is 1/2 mean over pixels and
channels of (L_student - L_teacher)^2; torch autograd in float64 supplies
its exact derivative with respect to the hash table and all MLP weights.
Sampled directions are constants of the estimator: w'_ij is drawn about
the detached n'_i.  Pins: central finite differences of this forward
(tests/test_oracle_render.py).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional

import numpy as np
import torch

from . import hashgrid, mis, mlp, sampling, shading


@dataclasses.dataclass(frozen=True)
class Options:
    n_dirs: int
    m_dirs: int = 8
    levels: int = 16
    log2_T: int = 19
    base_res: int = 16
    max_res: int = 2048
    near: float = 0.05
    far: float = 1.5
    f0: float = shading.F0_DEFAULT
    lambert: bool = False
    force_vis: float = -1.0      # < 0: use I's visibility
    force_vis2: float = -1.0
    hard_vis: bool = False       # v, v' = 1[sigma(z0) > 0.5] (Sec. 3.2 overview)
    sampling: str = "cosine"     # primary directions: 'cosine' or 'mis' (light + GGX, balance heuristic; mis.py)
    decision_arith: str = "fp64"  # arithmetic of the hard decisions: 'fp64', 'fp32' or 'bf16'
    flip_margin: float = 0.0     # > 0: also return the flip allowance of rows with |z0| < margin
    mis_margin: float = 0.0      # > 0 (MIS): also return the allowance of directions within this angle of a texel edge
    dir_seed: int = 0x5EED
    dense_coarse: bool = True
    # conditioning probe: relative Gaussian jitter of the secondary points x'
    # (0 = off), keyed by (jitter_seed, pixel id); used only to measure how
    # strongly the exact result reacts to float32-sized rounding of x'.
    x2_jitter: float = 0.0
    s_jitter: float = 0.0        # absolute jitter of the sphere points s of both samplers
    mlp_jitter: float = 0.0      # relative jitter of MLP inputs and hidden activations
    jitter_seed: int = 0

    @staticmethod
    def from_config(cfg, **kw) -> "Options":
        return Options(n_dirs=cfg.n_dirs, m_dirs=cfg.m_dirs, levels=cfg.levels,
                       log2_T=cfg.log2_T, base_res=cfg.base_res, max_res=cfg.max_res,
                       near=cfg.near, far=cfg.far, f0=cfg.f0, dir_seed=cfg.dir_seed, **kw)


@dataclasses.dataclass
class Params:
    """Float64 model parameters (may require grad)."""
    table: torch.Tensor                 # [L, T, F]
    brdf: list                          # [(W, b)] x 3
    irt: list
    env: torch.Tensor                   # [H, W, 4]

    @staticmethod
    def from_arrays(table, brdf_layers, irt_layers, env, requires_grad=False) -> "Params":
        t = torch.tensor(np.asarray(table, np.float64), requires_grad=requires_grad)
        b = [(torch.tensor(np.asarray(w, np.float64), requires_grad=requires_grad),
              torch.tensor(np.asarray(c, np.float64), requires_grad=requires_grad))
             for w, c in brdf_layers]
        i = [(torch.tensor(np.asarray(w, np.float64), requires_grad=requires_grad),
              torch.tensor(np.asarray(c, np.float64), requires_grad=requires_grad))
             for w, c in irt_layers]
        return Params(t, b, i, torch.tensor(np.asarray(env, np.float64)))


def _gbuffer_tensors(gb: Dict[str, np.ndarray], rows: np.ndarray):
    """(x, n, w_o, albedo, roughness) of G-buffer rows in float64.

    The paper's n and w_o are unit vectors; the G-buffer holds them rounded
    to float32, so the oracle takes the unit vectors those triples denote
    (normalised in float64).
    """
    def g(key, k):
        return torch.from_numpy(np.asarray(gb[key][rows, :k], np.float64))

    def unit(v):
        return v / v.norm(dim=-1, keepdim=True).clamp(min=1e-300)
    ar = torch.from_numpy(np.asarray(gb["albedo_rough"][rows], np.float64))
    return g("pos", 3), unit(g("normal", 3)), unit(g("view", 3)), ar[:, :3], ar[:, 3]


def _primary_dirs(x, n, wo, rough, q, prm: Params, opt: Options, jitter=None):
    """Primary directions w_i [P, N, 3] and their Eq. 1 weights relative to cosine sampling.

    Cosine sampling: the weight is None ((w . n) / p = pi).  MIS: the factor
    (n . w)+ / (n_L p_L + n_G p_G) times N / pi, so that (pi / N) sum stays the
    estimator's form.  With opt.mis_margin > 0 also returns how far that factor
    can move when p_L is read from a texel next to the direction's own (for
    directions within the margin of a texel edge), else None.  `jitter` [P, N, 3] (conditioning probe only) is added to
    the sphere point of a cosine sample or to an MIS direction.
    """
    N, M = opt.n_dirs, opt.m_dirs
    u1, u2 = sampling.uniforms(opt.dir_seed, sampling.counters(q, 0, M))
    if opt.sampling == "cosine":
        return sampling.cosine_direction(n[:, None, :], u1, u2, jitter), None, None
    marg, cond = mis.env_cdf(prm.env.detach().numpy()[..., :3].astype(np.float32))
    w, fac = mis.primary_directions(n, wo, rough, u1, u2, N, marg, cond)
    if jitter is not None:
        # the GGX visible-normal map amplifies the rounding of its own arithmetic near the
        # rim of its disk, so the probe also moves the uniforms of GGX draws (their map is
        # continuous; the light draws' CDF inversion is a decision both sides take alike)
        g_rows = ((n * wo).sum(-1) > mis.NOV_MIN)[:, None] & torch.from_numpy((np.arange(N) % 2 == 1)[None, :])
        lim = 1.0 - 2.0 ** -24
        w_g = mis.sample_ggx(n[:, None, :].expand_as(w), wo[:, None, :].expand_as(w),
                             (rough * rough)[:, None].expand(w.shape[:2]),
                             (u1 + jitter[..., 0]).clamp(0.0, lim), (u2 + jitter[..., 1]).clamp(0.0, lim))
        w = torch.where(g_rows[..., None], w_g, w)
        w = w + jitter
        w = w / w.norm(dim=-1, keepdim=True)
        nv = n[:, None, :].expand_as(w)
        wv = wo[:, None, :].expand_as(w)
        alpha = (rough * rough)[:, None].expand(w.shape[:2])
        n_g = torch.where((n * wo).sum(-1) > mis.NOV_MIN, torch.full_like(rough, N // 2),
                          torch.zeros_like(rough))[:, None]
        den = (N - n_g) * mis.pdf_light(w, marg, cond) + n_g * mis.pdf_ggx(w, nv, wv, alpha)
        fac = torch.clamp((nv * w).sum(-1), min=0.0) / den
    dfac = None
    if opt.mis_margin > 0:
        nv = n[:, None, :].expand_as(w)
        wv = wo[:, None, :].expand_as(w)
        alpha = (rough * rough)[:, None].expand(w.shape[:2])
        n_g = torch.where((n * wo).sum(-1) > mis.NOV_MIN, torch.full_like(rough, N // 2),
                          torch.zeros_like(rough))[:, None]
        den = (N - n_g) * mis.pdf_light(w, marg, cond) + n_g * mis.pdf_ggx(w, nv, wv, alpha)
        dp = (N - n_g) * mis.pdf_light_neighbours(w, marg, cond, opt.mis_margin)
        cos = torch.clamp((nv * w).sum(-1), min=0.0)
        # |cos / (den - dp) - cos / den| bounds the change when the density moves by at most dp
        dfac = cos * dp / (den * torch.clamp(den - dp, min=1e-300)) * (N / math.pi)
    return w, fac * (N / math.pi), dfac


def _kernel_logits(x, n, wo, rough, q, prm: Params, opt: Options, res, dense):
    """Visibility logits z0 [P, N] and z0' [P*N, M] as a kernel computes them.

    The chain that leads to the decisions (f, I, the bounce, f', B, the
    secondary directions, I again) is re-evaluated in opt.decision_arith:
    the table as the kernel reads it (FP16 for 'bf16'), x' rounded to
    float32, cell fractions as the kernel takes them (from float32 g for the
    BF16 secondary encode, exact otherwise), the features rounded to the MLP
    input format,
    and the MLPs in mlp3_arith (for 'bf16', the primary evaluation of I in
    the split form 'bf16x3': there the kernel feeds the float32 features).
    Directions and depth are float64.
    """
    arith = opt.decision_arith
    P, N, M = x.shape[0], opt.n_dirs, opt.m_dirs
    w_i, _, _ = _primary_dirs(x, n, wo, rough, q, prm, opt)                # unjittered, [P, N, 3]
    tab = mlp.round_to(prm.table, "fp16" if arith == "bf16" else "fp32")
    feat = lambda f: mlp.round_to(f, "bf16" if arith == "bf16" else "fp32")
    # the fused kernels take cell fractions from the exact grid coordinate (float64 here) for the
    # primary encode, and for the secondary one in FP32; the BF16 secondary encode uses float32 g
    f32 = mlp.round_to(hashgrid.encode(x, tab, res, dense), "fp32")
    f = f32 if arith == "bf16" else feat(f32)
    f_rep = f[:, None, :].expand(P, N, f.shape[1]).reshape(P * N, -1)
    # the BF16 kernels evaluate I at the primary point in split precision (hi + lo bf16 parts)
    y = mlp.mlp3_arith(torch.cat([f_rep, mlp.positional_encoding(w_i.reshape(P * N, 3))], dim=-1), prm.irt,
                       "bf16x3" if arith == "bf16" else arith)
    t = mlp.depth_from_logit(torch.nn.functional.softplus(y[:, 1]), opt.near, opt.far)
    x2 = x[:, None, :] + t.reshape(P, N, 1) * w_i
    f2 = feat(hashgrid.encode(mlp.round_to(x2.reshape(P * N, 3), "fp32"), tab, res, dense, fp32_grid=arith == "bf16"))
    yb = mlp.mlp3_arith(f2, prm.brdf, arith)
    n2 = yb[:, 0:3] / yb[:, 0:3].norm(dim=1, keepdim=True).clamp(min=1e-12)
    slots = 1 + np.arange(M, dtype=np.uint64)
    u1, u2 = sampling.uniforms(opt.dir_seed, sampling.counters(q.reshape(-1, 1), slots[None, :], M))
    w_j = sampling.cosine_direction(n2[:, None, :], u1, u2)
    f2_rep = f2[:, None, :].expand(P * N, M, f2.shape[1]).reshape(P * N * M, -1)
    z2 = mlp.mlp3_arith(torch.cat([f2_rep, mlp.positional_encoding(w_j.reshape(-1, 3))], dim=-1), prm.irt, arith)
    return y[:, 0].reshape(P, N), z2[:, 0].reshape(P * N, M)


def render_points(x, n, wo, albedo, rough, global_ids: np.ndarray, prm: Params, opt: Options,
                  fixed_dirs: Optional[torch.Tensor] = None, want_dirs: bool = False,
                  decide: Optional[Params] = None):
    """Radiance [P, 3] of P primary points with global pixel ids (RNG keys).

    decide: the parameters the hard decisions are taken with (default prm);
    the conditioning probe passes the unperturbed ones so that its jittered
    renders keep the decisions of the render they are compared with.  With
    opt.hard_vis and opt.flip_margin > 0 returns (radiance, allowance [P, 3]).
    """
    P, N, M = x.shape[0], opt.n_dirs, opt.m_dirs
    res = hashgrid.level_resolutions(opt.levels, opt.base_res, opt.max_res)
    dense = hashgrid.dense_levels(res, 1 << opt.log2_T, opt.dense_coarse)

    # (a) primary feature
    f = hashgrid.encode(x, prm.table, res, dense)
    jit = None
    if opt.mlp_jitter > 0:
        g = torch.Generator().manual_seed(int(opt.jitter_seed) * 1000003 + int(np.asarray(global_ids)[0]))
        jit = (opt.mlp_jitter, g)

    # primary directions, slot 0 of sample q = gid * N + i
    q = np.asarray(global_ids, np.uint64)[:, None] * np.uint64(N) + np.arange(N, dtype=np.uint64)[None, :]
    w_i, wfac, dfac = _primary_dirs(x, n, wo, rough, q, prm, opt, _jitter(opt, global_ids, 0, (N, 3)))  # [P, N, 3]

    # (c) visibility and depth along w_i
    f_rep = f[:, None, :].expand(P, N, f.shape[1]).reshape(P * N, -1)
    v, t = mlp.implicit_ray_tracer(f_rep, w_i.reshape(P * N, 3), prm.irt, opt.near, opt.far, jit)
    z0k = z2k = None
    if opt.hard_vis:
        if opt.decision_arith == "fp64":
            v = (v > 0.5).to(v.dtype)
        else:
            z0k, z2k = _kernel_logits(x, n, wo, rough, q, prm if decide is None else decide, opt, res, dense)
            v = (z0k.reshape(-1) > 0).to(v.dtype)
    if opt.force_vis >= 0:
        v = torch.full_like(v, opt.force_vis)

    # (d) bounce and re-encode
    x2 = x[:, None, :] + t.reshape(P, N, 1) * w_i                          # x' = x + t w
    if opt.x2_jitter > 0:
        x2 = x2 * (1.0 + opt.x2_jitter * _noise(opt, global_ids, 2, (N, 3)))
    f2 = hashgrid.encode(x2.reshape(P * N, 3), prm.table, res, dense)
    a2, r2, n2 = mlp.brdf_decoder(f2, prm.brdf, jit)                      # (b)

    # secondary directions, slots 1..M about the (detached) secondary normal
    if fixed_dirs is None:
        slots = 1 + np.arange(M, dtype=np.uint64)
        u1, u2 = sampling.uniforms(opt.dir_seed, sampling.counters(q.reshape(-1, 1), slots[None, :], M))
        w_j = sampling.cosine_direction(n2.detach()[:, None, :], u1, u2,
                                        _jitter(opt, global_ids, 1, (N, M, 3), flat=True))   # [P*N, M, 3]
    else:
        w_j = fixed_dirs
    f2_rep = f2[:, None, :].expand(P * N, M, f2.shape[1]).reshape(P * N * M, -1)
    v2, _ = mlp.implicit_ray_tracer(f2_rep, w_j.reshape(-1, 3), prm.irt, opt.near, opt.far, jit)
    v2 = v2.reshape(P * N, M)
    if opt.hard_vis:
        v2 = (v2 > 0.5).to(v2.dtype) if z2k is None else (z2k > 0).to(v2.dtype)
    if opt.force_vis2 >= 0:
        v2 = torch.full_like(v2, opt.force_vis2)

    # (e) secondary sum at x' towards -w_i (Eq. 1 at x')
    wo2 = -w_i.reshape(P * N, 1, 3)
    fr2 = shading.brdf(a2[:, None, :], r2[:, None], n2[:, None, :], w_j, wo2, opt.f0, opt.lambert)
    le2 = shading.env_lookup(prm.env, w_j)
    lo2 = shading.mc_sum(v2[..., None] * le2 * fr2, M).reshape(P, N, 3)

    # Eq. 2, then Eq. 1 at x
    v = v.reshape(P, N, 1)
    le1 = shading.env_lookup(prm.env, w_i)
    li = v * le1 + (1.0 - v) * lo2
    fr1 = shading.brdf(albedo[:, None, :], rough[:, None], n[:, None, :], w_i, wo[:, None, :],
                       opt.f0, opt.lambert)
    base_term = li * fr1
    if wfac is not None:
        fr1 = fr1 * wfac[..., None]
    out = shading.mc_sum(li * fr1, N)
    allow_mis = None
    if dfac is not None:
        allow_mis = shading.mc_sum(base_term.abs() * dfac[..., None], N)
    if opt.hard_vis and opt.flip_margin > 0:
        if z0k is None:
            raise ValueError("flip_margin needs a kernel decision_arith")
        amb1 = (z0k.abs() < opt.flip_margin).to(out.dtype)[..., None]                  # [P, N, 1]
        amb2 = (z2k.abs() < opt.flip_margin).to(out.dtype)[..., None]                  # [P*N, M, 1]
        if opt.force_vis >= 0:
            amb1 = torch.zeros_like(amb1)
        if opt.force_vis2 >= 0:
            amb2 = torch.zeros_like(amb2)
        # a flipped v swaps L_env(w_i) and L'_o,i; a flipped v' adds or removes its term of L'_o,i,
        # which reaches the pixel unless v = 1 is certain
        d_sec = shading.mc_sum(amb2 * (le2 * fr2).abs(), M).reshape(P, N, 3)
        reach = torch.maximum(1.0 - v, amb1)
        allow = shading.mc_sum((amb1 * (le1 - lo2).abs() + reach * d_sec) * fr1.abs(), N)
        if allow_mis is not None:
            allow = allow + allow_mis
        return out, allow
    if allow_mis is not None:
        return out, allow_mis
    if want_dirs:
        return out, w_j.detach()
    return out


def _noise(opt: Options, global_ids, stream: int, shape) -> torch.Tensor:
    return torch.from_numpy(np.stack([np.random.default_rng([opt.jitter_seed, stream, int(g)]).standard_normal(shape)
                                      for g in np.asarray(global_ids)]))


def _jitter(opt: Options, global_ids, stream: int, shape, flat: bool = False):
    if opt.s_jitter <= 0:
        return None
    z = opt.s_jitter * _noise(opt, global_ids, stream, shape)
    return z.reshape(-1, *shape[1:]) if flat else z


def render(gb: Dict[str, np.ndarray], prm: Params, opt: Options, pixel_offset: int = 0,
           rows: Optional[np.ndarray] = None, chunk_rows: int = 1 << 17, decide: Optional[Params] = None):
    """Radiance [len(rows), 3] (float64) of G-buffer rows (default: all).

    The RNG key of row p is pixel_offset + p, so a frame rendered in pieces
    equals the frame rendered at once.  With opt.hard_vis and
    opt.flip_margin > 0 returns (radiance, flip allowance), both [len(rows), 3].
    """
    P = gb["pos"].shape[0]
    rows = np.arange(P) if rows is None else np.asarray(rows)
    per = max(1, chunk_rows // (opt.n_dirs * opt.m_dirs))
    pair = (opt.hard_vis and opt.flip_margin > 0) or (opt.sampling == "mis" and opt.mis_margin > 0)
    out, allow = [], []
    with torch.no_grad():
        for s in range(0, rows.size, per):
            r = rows[s:s + per]
            res = render_points(*_gbuffer_tensors(gb, r), pixel_offset + r, prm, opt, decide=decide)
            if pair:
                out.append(res[0].numpy())
                allow.append(res[1].numpy())
            else:
                out.append(res.numpy())
    cat = lambda xs: np.concatenate(xs, axis=0) if xs else np.zeros((0, 3))
    return (cat(out), cat(allow)) if pair else cat(out)


def float32_sensitivity(gb: Dict[str, np.ndarray], prm: Params, opt: Options, pixel_offset: int = 0,
                        rows: Optional[np.ndarray] = None, rel: float = 2.0 ** -23, draws: int = 2,
                        mlp: bool = False, table_rel: float = 2.0 ** -11) -> np.ndarray:
    """Per-pixel, per-channel max |L(jittered) - L| over `draws` float32-sized jitters.

    Two inputs of the exact result are ill-conditioned at float32 scale:
    the secondary points x' = x + t w feed the finest hash levels, whose
    features change by up to ~N_l * |table step| per unit of x'; and a
    grazing direction normalize(n + s) moves by |ds| / |n + s| when n + s is
    short.  A pixel dominated by such a sample under a sharp specular lobe
    can move by far more than 1e-4 when x' or s changes by one float32
    rounding.  This probe jitters x' (relative) and s (absolute) by `rel`
    and reports how far the exact result moves; the FP32 parity tests scale
    their per-pixel bound by it.  With mlp=True it also jitters the MLP inputs
    and hidden activations (per sample) and both hidden weight matrices (per
    draw) by `rel`, and the table by `table_rel` (2^-11: the roundings of a
    bf16 MLP with an FP16 table, used by the BF16 tests; 0 for a float32
    table, which both sides read exactly).
    """
    opt = dataclasses.replace(opt, flip_margin=0.0, mis_margin=0.0)
    decide = prm if (opt.hard_vis and opt.decision_arith != "fp64") else None   # decisions stay those of base
    base = render(gb, prm, opt, pixel_offset, rows)
    worst = np.zeros_like(base)
    for d in range(draws):
        o = dataclasses.replace(opt, x2_jitter=rel, s_jitter=rel, mlp_jitter=rel if mlp else 0.0, jitter_seed=1 + d)
        p = _perturbed_weights(prm, rel, 1 + d, table_rel) if mlp else prm
        worst = np.maximum(worst, np.abs(render(gb, p, o, pixel_offset, rows, decide=decide) - base))
    return worst


def _perturbed_weights(prm: Params, rel: float, seed: int, table_rel: float = 2.0 ** -11) -> Params:
    """Params with both hidden layers' weight matrices scaled by (1 + rel z) and the
    table by (1 + table_rel z): the systematic part of bf16 weights and an FP16 table."""
    g = torch.Generator().manual_seed(seed)

    def jw(layers):
        out = []
        for k, (w, b) in enumerate(layers):
            if k < 2:
                w = w * (1.0 + rel * torch.randn(w.shape, generator=g, dtype=w.dtype))
            out.append((w, b))
        return out
    table = prm.table * (1.0 + table_rel * torch.randn(prm.table.shape, generator=g, dtype=prm.table.dtype))
    return Params(table, jw(prm.brdf), jw(prm.irt), prm.env)


def distill_loss(gb, rows, student: Params, target: torch.Tensor, opt: Options,
                 pixel_offset: int = 0, fixed_dirs=None, want_dirs=False):
    """1/2 mean over rays and channels of (L_student - L_teacher)^2."""
    r = np.asarray(rows)
    out = render_points(*_gbuffer_tensors(gb, r), pixel_offset + r, student, opt,
                        fixed_dirs=fixed_dirs, want_dirs=want_dirs)
    if want_dirs:
        out, dirs = out
    loss = 0.5 * ((out - target) ** 2).mean()
    return (loss, dirs) if want_dirs else loss


def distill_gradient(gb, rows, student: Params, target: torch.Tensor, opt: Options,
                     pixel_offset: int = 0):
    """FP64 loss and its gradient w.r.t. the table and both MLPs' packed weights."""
    for p in _leaves(student):
        p.grad = None
    loss = distill_loss(gb, rows, student, target, opt, pixel_offset)
    loss.backward()
    g_table = student.table.grad.clone()
    g_brdf = torch.cat([t.grad.reshape(-1) for wb in student.brdf for t in wb])
    g_irt = torch.cat([t.grad.reshape(-1) for wb in student.irt for t in wb])
    return float(loss.detach()), g_table, g_brdf, g_irt


def upstream_gradient(student_rad: np.ndarray, target_rad: np.ndarray) -> np.ndarray:
    """dLoss/dL_student for the distillation loss: (L_s - L_t) / (3 P) per channel."""
    return (student_rad - target_rad) / (3.0 * student_rad.shape[0])


def _leaves(p: Params):
    yield p.table
    for w, b in p.brdf + p.irt:
        yield w
        yield b


def secondary_samples_per_second(opt: Options, n_pixels: int, seconds: float) -> float:
    return n_pixels * opt.n_dirs / seconds

