"""Pins of the oracle's whole path (Eq. 1, Eq. 2, the bounce) and of its FP64 gradient."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import scenegen
from oracle import render, shading

SMALL = scenegen.SceneConfig("small", 4, 4, 8, m_dirs=4, levels=6, log2_T=10, base_res=4, max_res=64,
                             env_h=8, env_w=16)


def _setup(cfg=SMALL, seed=0, bias=0.0, white=False, env_rgb=None):
    sc = scenegen.make_scene(cfg, seed, bias_scale=bias)
    env = sc.env.copy()
    if white:
        env[..., :3] = 1.0
    if env_rgb is not None:
        env[..., :3] = np.asarray(env_rgb)
    gb = scenegen.make_gbuffer(cfg.n_pixels, seed)
    prm = render.Params.from_arrays(sc.table, sc.brdf, sc.irt, env)
    return gb, prm


def _opt(cfg=SMALL, **kw):
    return render.Options.from_config(cfg, **kw)


def test_white_furnace_returns_albedo():
    # L_env = 1, V = 1, Lambert: (pi/N) sum_i (a/pi) = a exactly (the spec furnace test)
    gb, prm = _setup(white=True)
    out = render.render(gb, prm, _opt(force_vis=1.0, lambert=True))
    np.testing.assert_allclose(out, gb["albedo_rough"][:, :3], rtol=1e-13)


def test_coloured_constant_env_scales_albedo():
    gb, prm = _setup(env_rgb=[0.5, 2.0, 3.0])
    out = render.render(gb, prm, _opt(force_vis=1.0, lambert=True))
    np.testing.assert_allclose(out, gb["albedo_rough"][:, :3] * [0.5, 2.0, 3.0], rtol=1e-13)


def test_fully_occluded_is_black():
    gb, prm = _setup()
    out = render.render(gb, prm, _opt(force_vis=0.0, force_vis2=0.0))
    assert np.all(out == 0.0)


def test_one_bounce_closed_form():
    # V = 0, V' = 1, white env, Lambert and a decoder whose output is its bias b3:
    # every x' has albedo a' = sigmoid(b3[3:6]), so L = a * a' exactly (Eq. 2 with V = 0).
    cfg = SMALL
    sc = scenegen.make_scene(cfg, 1)
    b3 = np.array([0.3, -0.2, 0.9, 0.4, -1.0, 2.0, 0.1], np.float32)
    brdf = [(w * 0, b * 0) for w, b in sc.brdf[:2]] + [(sc.brdf[2][0] * 0, b3)]
    env = sc.env.copy()
    env[..., :3] = 1.0
    gb = scenegen.make_gbuffer(cfg.n_pixels, 1)
    prm = render.Params.from_arrays(sc.table, brdf, sc.irt, env)
    out = render.render(gb, prm, _opt(force_vis=0.0, force_vis2=1.0, lambert=True))
    a2 = 1.0 / (1.0 + np.exp(-b3[3:6].astype(np.float64)))
    np.testing.assert_allclose(out, gb["albedo_rough"][:, :3] * a2, rtol=1e-12)


def test_eq2_is_linear_in_visibility():
    # L(v) = v * L(v=1) + (1 - v) * L(v=0) for a constant v (Eq. 2 is a convex blend)
    gb, prm = _setup(bias=0.3)
    l1 = render.render(gb, prm, _opt(force_vis=1.0))
    l0 = render.render(gb, prm, _opt(force_vis=0.0))
    lv = render.render(gb, prm, _opt(force_vis=0.3))
    np.testing.assert_allclose(lv, 0.3 * l1 + 0.7 * l0, rtol=1e-12)


def test_sharded_frame_equals_whole_frame():
    gb, prm = _setup(bias=0.1)
    opt = _opt()
    whole = render.render(gb, prm, opt)
    rows = np.arange(SMALL.n_pixels)
    parts = [render.render({k: v[r] for k, v in gb.items()}, prm, opt, pixel_offset=int(r[0]))
             for r in np.array_split(rows, 3)]
    np.testing.assert_array_equal(np.concatenate(parts), whole)
    sub = render.render(gb, prm, opt, rows=np.array([5, 2, 11]))
    np.testing.assert_array_equal(sub, whole[[5, 2, 11]])


def test_direct_term_converges_to_directional_albedo():
    # V = 1, L_env = 1: the primary sum estimates int f_r (w.n) dw, here compared with
    # midpoint quadrature over the hemisphere (a check of the pi/N weighting and pdf).
    cfg = dataclasses.replace(SMALL, n_dirs=8192)
    gb, prm = _setup(cfg, white=True)
    rows = np.array([0, 3, 6])
    ar = gb["albedo_rough"]
    ar[rows, 3] = [0.35, 0.6, 1.0]
    # a view 37 degrees off the normal keeps the estimator's variance moderate
    for r in rows:
        n = gb["normal"][r, :3].astype(np.float64)
        t = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 else [0.0, 1.0, 0.0])
        t /= np.linalg.norm(t)
        gb["view"][r, :3] = 0.8 * n + 0.6 * t
    out = render.render(gb, prm, render.Options.from_config(cfg, force_vis=1.0), rows=rows)
    nt, nphi = 600, 1200
    th = (np.arange(nt) + 0.5) * (np.pi / 2) / nt
    ph = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    T, P = np.meshgrid(th, ph, indexing="ij")
    for k, r in enumerate(rows):
        n = gb["normal"][r, :3].astype(np.float64)
        a = np.cross(n, [1.0, 0, 0] if abs(n[0]) < 0.9 else [0, 1.0, 0])
        a /= np.linalg.norm(a)
        b = np.cross(n, a)
        d = (np.sin(T)[..., None] * (np.cos(P)[..., None] * a + np.sin(P)[..., None] * b)
             + np.cos(T)[..., None] * n)
        fr = shading.brdf(torch.from_numpy(ar[r, :3].astype(np.float64)), torch.tensor(float(ar[r, 3]), dtype=torch.float64),
                          torch.from_numpy(n), torch.from_numpy(d),
                          torch.from_numpy(gb["view"][r, :3].astype(np.float64))).numpy()
        quad = (fr * (np.cos(T) * np.sin(T))[..., None]).sum((0, 1)) * (np.pi / 2 / nt) * (2 * np.pi / nphi)
        # the estimator's standard error at 8192 samples is below 0.25 % for these lobes
        np.testing.assert_allclose(out[k], quad, rtol=0.015)


def _grad_setup():
    cfg = dataclasses.replace(SMALL, n_dirs=4, m_dirs=2, levels=4, log2_T=8, base_res=4, max_res=32)
    sc = scenegen.make_scene(cfg, 2, bias_scale=0.2)
    teacher = scenegen.make_scene(cfg, 1, bias_scale=0.2)
    gb = scenegen.make_gbuffer(cfg.n_pixels, 3)
    opt = render.Options.from_config(cfg)
    rows = np.arange(6)
    t_prm = render.Params.from_arrays(teacher.table, teacher.brdf, teacher.irt, sc.env)
    with torch.no_grad():
        target = torch.from_numpy(render.render(gb, t_prm, opt, rows=rows))
    s_prm = render.Params.from_arrays(sc.table, sc.brdf, sc.irt, sc.env, requires_grad=True)
    return gb, rows, s_prm, target, opt


def test_gradient_matches_central_differences():
    gb, rows, prm, target, opt = _grad_setup()
    loss, dirs = render.distill_loss(gb, rows, prm, target, opt, want_dirs=True)
    loss.backward()
    rng = np.random.default_rng(0)
    leaves = list(render._leaves(prm))
    checked = 0
    for leaf in leaves:
        g = leaf.grad.reshape(-1)
        # prefer entries that matter (the table is sparse in its gradient)
        nz = torch.nonzero(g).reshape(-1).numpy()
        pick = rng.choice(nz, size=min(6, nz.size), replace=False) if nz.size else []
        for idx in pick:
            def f(delta):
                with torch.no_grad():
                    flat = leaf.view(-1)
                    old = float(flat[idx])
                    flat[idx] = old + delta
                    val = float(render.distill_loss(gb, rows, prm, target, opt, fixed_dirs=dirs))
                    flat[idx] = old
                return val
            # central differences at eps = 1e-3, 5e-4, 2.5e-4: in the smooth regime the
            # error of the finest one is below the gap between the last two
            eps = 1e-3
            fds = [(f(e) - f(-e)) / (2 * e) for e in (eps, eps / 2, eps / 4)]
            gap = abs(fds[1] - fds[2])
            if gap > 1e-4 * max(abs(fds[2]), 1e-12) + 1e-15:
                continue        # a kink (ReLU, clamp or cell crossing) inside the stencil
            tol = max(1e-6 * abs(fds[2]), 2.0 * gap) + 1e-13
            assert abs(float(g[idx]) - fds[2]) <= tol, (leaf.shape, idx, float(g[idx]), fds)
            checked += 1
    assert checked >= 30


# ---- hard visibility (the paper's inference, Sec. 3.2 overview) -------------

def _scaled_visibility_row(prm, scale=None, const=None):
    """Copy of prm with I's output row 0 (the visibility logit z0) scaled, or set to a constant."""
    (w1, b1), (w2, b2), (w3, b3) = prm.irt
    w3, b3 = w3.clone(), b3.clone()
    if scale is not None:
        w3[0] *= scale
        b3[0] *= scale
    if const is not None:
        w3[0] = 0.0
        b3[0] = const
    return dataclasses.replace(prm, irt=[(w1, b1), (w2, b2), (w3, b3)])


def test_hard_visibility_ignores_a_positive_scale_of_the_logit():
    # v = 1[sigmoid(z0) > 0.5] depends on the sign of z0 only; the soft blend does not
    gb, prm = _setup(bias=0.2)
    prm7 = _scaled_visibility_row(prm, scale=7.5)
    hard, hard7 = (render.render(gb, p, _opt(hard_vis=True)) for p in (prm, prm7))
    np.testing.assert_array_equal(hard, hard7)
    soft, soft7 = (render.render(gb, p, _opt()) for p in (prm, prm7))
    assert np.max(np.abs(soft - soft7)) > 1e-3


def test_hard_visibility_is_the_saturated_sigmoid():
    # the soft path with z0 scaled by 1e9 has sigmoid(z0) in {0, 1} exactly in float64, for v and v'
    gb, prm = _setup(bias=0.2)
    hard = render.render(gb, prm, _opt(hard_vis=True))
    soft_sat = render.render(gb, _scaled_visibility_row(prm, scale=1e9), _opt())
    np.testing.assert_allclose(hard, soft_sat, rtol=1e-12, atol=1e-15)
    assert np.max(np.abs(hard - render.render(gb, prm, _opt()))) > 1e-3


@pytest.mark.parametrize("z0, forced", [(0.5, dict(force_vis=1.0)), (-0.5, dict(force_vis=0.0, force_vis2=0.0))])
def test_hard_visibility_with_a_constant_logit(z0, forced):
    # z0 > 0 everywhere: every direction is visible, nothing bounces (the direct term alone);
    # z0 < 0 everywhere: every direction is a shadow ray whose secondary directions are all occluded
    gb, prm = _setup(bias=0.2)
    hard = render.render(gb, _scaled_visibility_row(prm, const=z0), _opt(hard_vis=True))
    ref = render.render(gb, prm, _opt(**forced))
    np.testing.assert_allclose(hard, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("arith, tol", [("fp32", 1e-5), ("bf16", 2e-2)])
def test_kernel_logits_follow_the_float64_chain(arith, tol):
    # the decision chain re-evaluated in a kernel's arithmetic stays within that
    # arithmetic's rounding of the float64 chain (I at x, the bounce, B, I at x').
    # Secondary logits inherit the conditioning of x' (one rounding of t can move x'
    # across fine-level texels), so they are held to the bound on 95 % of the rows.
    from oracle import hashgrid, mlp, sampling
    cfg = SMALL
    gb, prm = _setup(bias=0.2)
    opt = _opt(hard_vis=True, decision_arith=arith)
    rows = np.arange(cfg.n_pixels)
    x, n, wo, alb, rough = render._gbuffer_tensors(gb, rows)
    res = hashgrid.level_resolutions(opt.levels, opt.base_res, opt.max_res)
    dense = hashgrid.dense_levels(res, 1 << opt.log2_T, opt.dense_coarse)
    N, M = opt.n_dirs, opt.m_dirs
    q = rows.astype(np.uint64)[:, None] * np.uint64(N) + np.arange(N, dtype=np.uint64)[None, :]
    z0k, z2k = render._kernel_logits(x, n, wo, rough, q, prm, opt, res, dense)
    # the float64 chain, written out from the oracle's stage functions
    u1, u2 = sampling.uniforms(opt.dir_seed, sampling.counters(q, 0, M))
    w_i = sampling.cosine_direction(n[:, None, :], u1, u2)
    f = hashgrid.encode(x, prm.table, res, dense)
    f_rep = f[:, None, :].expand(-1, N, -1).reshape(-1, f.shape[1])
    y = mlp.mlp3(torch.cat([f_rep, mlp.positional_encoding(w_i.reshape(-1, 3))], -1), prm.irt)
    t = mlp.depth_from_logit(torch.nn.functional.softplus(y[:, 1]), opt.near, opt.far)
    x2 = (x[:, None, :] + t.reshape(-1, N, 1) * w_i).reshape(-1, 3)
    f2 = hashgrid.encode(x2, prm.table, res, dense)
    _, _, n2 = mlp.brdf_decoder(f2, prm.brdf)
    u1, u2 = sampling.uniforms(opt.dir_seed, sampling.counters(q.reshape(-1, 1), 1 + np.arange(M, dtype=np.uint64)[None, :], M))
    w_j = sampling.cosine_direction(n2[:, None, :], u1, u2)
    f2_rep = f2[:, None, :].expand(-1, M, -1).reshape(-1, f2.shape[1])
    z2 = mlp.mlp3(torch.cat([f2_rep, mlp.positional_encoding(w_j.reshape(-1, 3))], -1), prm.irt)[:, 0]
    scale = float(y[:, 0].abs().max())
    assert float((z0k.reshape(-1) - y[:, 0]).abs().max()) <= tol * scale
    assert float(np.quantile((z2k.reshape(-1) - z2).abs().numpy(), 0.95)) <= tol * scale
    # and the decisions agree wherever the float64 logit is clear of the rounding
    clear = y[:, 0].abs() > tol * scale
    assert bool(((z0k.reshape(-1) > 0) == (y[:, 0] > 0))[clear].all())


def test_hard_flip_allowance_covers_the_float64_decisions():
    # decisions taken in bf16 arithmetic and in float64 differ only on rows within the
    # margin, so the float64 hard frame lies within the bf16 frame's flip allowance
    gb, prm = _setup(bias=0.2)
    hard64 = render.render(gb, prm, _opt(hard_vis=True))
    hard16, allow = render.render(gb, prm, _opt(hard_vis=True, decision_arith="bf16", flip_margin=0.1))
    assert np.all(np.abs(hard64 - hard16) <= allow + 1e-12)
    assert np.all(allow >= 0)
    # the bf16-decided frame keeps the scale invariance of the hit test (a power-of-two scale is exact)
    hard16s = render.render(gb, _scaled_visibility_row(prm, scale=4.0), _opt(hard_vis=True, decision_arith="bf16"))
    np.testing.assert_array_equal(hard16s, hard16)
