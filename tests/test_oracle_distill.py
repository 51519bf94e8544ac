"""Pins of the oracle's per-head distillation (Sec. 3.3) and its Adam step."""
import math

import numpy as np
import pytest
import torch

import scenegen
from oracle import distill, render

CFG = scenegen.SceneConfig("d", 4, 1, 16, levels=6, log2_T=10, base_res=4, max_res=64)


def _batch(R=4, K=16, seed=0):
    gb = scenegen.make_gbuffer(R, seed)
    x = torch.from_numpy(gb["pos"][:, :3].astype(np.float64))
    n = torch.from_numpy(gb["normal"][:, :3].astype(np.float64))
    w = distill.stratified_sphere(np.arange(R), K, 0x5EED)
    return x, n, w


def _params(seed):
    sc = scenegen.make_scene(CFG, seed, bias_scale=0.1)
    return render.Params.from_arrays(sc.table, sc.brdf, sc.irt, sc.env)


def test_one_direction_per_stratum():
    K, S = 64, 8
    w = distill.stratified_sphere(np.arange(3), K, 7)
    u1 = (1.0 - w[..., 2]) / 2.0
    u2 = torch.remainder(torch.atan2(w[..., 1], w[..., 0]), 2 * math.pi) / (2 * math.pi)
    cell = torch.floor(u1 * S) * S + torch.floor(u2 * S)
    for r in range(3):
        assert sorted(cell[r].long().tolist()) == list(range(K))
    np.testing.assert_allclose(w.norm(dim=-1).numpy(), 1.0, atol=1e-12)


def test_bce_and_l1_closed_forms():
    z = torch.tensor([0.0, 2.0, -3.0, 40.0], dtype=torch.float64)
    y = torch.tensor([1.0, 0.0, 1.0, 1.0], dtype=torch.float64)
    # -log sigmoid(z) = log(1 + e^-z) for y = 1, -log(1 - sigmoid(z)) = log(1 + e^z) for y = 0
    ref = np.where(y.numpy() > 0, np.logaddexp(0.0, -z.numpy()), np.logaddexp(0.0, z.numpy()))
    np.testing.assert_allclose(distill.bce_with_logits(z, y).numpy(), ref, rtol=1e-12)
    assert float(distill.bce_with_logits(z[:1], y[:1])) == pytest.approx(math.log(2.0), rel=1e-15)


def test_identical_student_and_teacher():
    # the L1 terms vanish and BCE against the binarised own visibility is softplus(-|z0|)
    x, n, w = _batch()
    opt = render.Options.from_config(CFG)
    prm = _params(3)
    tg = distill.teacher_targets(x, n, w, prm, opt, decision_arith="fp32")
    total, (lb, lc, ld) = distill.distill_loss(x, n, w, prm, tg, opt)
    assert float(lb) == 0.0 and float(ld) == 0.0
    _, z0, _ = distill._heads(x, w, prm, opt)
    front = ((w * n[:, None, :]).sum(-1) > 0).to(torch.float64)
    ref = sum(float((torch.nn.functional.softplus(-z0[r].abs()) * front[r]).sum() / front[r].sum())
              for r in range(x.shape[0])) / x.shape[0]
    assert float(lc) == pytest.approx(ref, rel=1e-9)


def test_gradient_matches_finite_differences():
    x, n, w = _batch(R=3, K=16, seed=1)
    opt = render.Options.from_config(CFG)
    student, teacher = _params(2), _params(1)
    tg = distill.teacher_targets(x, n, w, teacher, opt)
    _, g_tab, g_b, g_i = distill.distill_gradient(x, n, w, student, tg, opt)
    rng = np.random.default_rng(0)

    def loss_with(mutate):
        p = render.Params(student.table.clone(), [(a.clone(), b.clone()) for a, b in student.brdf],
                          [(a.clone(), b.clone()) for a, b in student.irt], student.env)
        mutate(p)
        return float(distill.distill_loss(x, n, w, p, tg, opt)[0])
    # a few I and B weights and the most-touched table entries; eps small against the L1 kinks
    checks = []
    for layer, (wt, _) in enumerate(student.irt[:2]):
        for _ in range(3):
            i, j = rng.integers(wt.shape[0]), rng.integers(wt.shape[1])
            checks.append(("irt", layer, i, j))
    for _ in range(3):
        i, j = rng.integers(student.brdf[1][0].shape[0]), rng.integers(student.brdf[1][0].shape[1])
        checks.append(("brdf", 1, i, j))
    off_i = [0, 64 * (student.irt[0][0].shape[1]) + 64]
    off_b = [0, 64 * (student.brdf[0][0].shape[1]) + 64]
    for kind, layer, i, j in checks:
        eps = 1e-6

        def mut(sign):
            def f(p):
                (p.irt if kind == "irt" else p.brdf)[layer][0][i, j] += sign * eps
            return f
        fd = (loss_with(mut(1)) - loss_with(mut(-1))) / (2 * eps)
        g = g_i if kind == "irt" else g_b
        off = (off_i if kind == "irt" else off_b)[layer]
        ncol = (student.irt if kind == "irt" else student.brdf)[layer][0].shape[1]
        assert float(g[off + i * ncol + j]) == pytest.approx(fd, rel=1e-4, abs=1e-9)
    flat = g_tab.reshape(-1, 2).norm(dim=1)
    for e in torch.argsort(flat, descending=True)[:3].tolist():
        l, t = divmod(e, student.table.shape[1])
        for c in range(2):
            def mt(sign):
                def f(p):
                    p.table[l, t, c] += sign * 1e-6
                return f
            fd = (loss_with(mt(1)) - loss_with(mt(-1))) / 2e-6
            assert float(g_tab[l, t, c]) == pytest.approx(fd, rel=1e-4, abs=1e-9)


def test_adam_step_closed_form():
    p, g = np.array([1.0, -2.0]), np.array([0.5, -0.25])
    p1, m1, v1 = distill.adam_step(p, g, np.zeros(2), np.zeros(2), 1, lr=0.1, weight_decay=0.0)
    # first step: m_hat = g, v_hat = g^2, so p moves by lr * sign(g) (up to eps)
    np.testing.assert_allclose(p1, p - 0.1 * np.sign(g), rtol=1e-7)
    p2, _, _ = distill.adam_step(p, g, np.zeros(2), np.zeros(2), 1, lr=0.1, weight_decay=1.0)
    np.testing.assert_allclose(p2, p - 0.1 * np.sign(g + p), rtol=1e-7)
