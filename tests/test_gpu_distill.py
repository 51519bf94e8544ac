"""Per-head distillation (rt_distill_dirs / rt_distill_backward / rt_adam_step) against the oracle."""
import numpy as np
import pytest
import torch

import scenegen
from oracle import distill as odist
from oracle import render as orender
from tests import helpers

pytestmark = pytest.mark.gpu

CFG = scenegen.SceneConfig("d", 40, 1, 16, levels=8, log2_T=14, base_res=16, max_res=256, env_h=16, env_w=32)


@pytest.fixture(scope="module")
def lib():
    from paper_2409_10327_gb300 import build
    build.build()
    from paper_2409_10327_gb300 import binding
    return binding


def _scene(seed):
    return scenegen.make_scene(CFG, seed, bias_scale=0.1)


def test_stratified_directions_match_oracle(lib):
    r = helpers.renderer_for(CFG, _scene(2))
    d = r.distill_dirs(5, 64, ray_offset=11).cpu().numpy()
    ref = odist.stratified_sphere(11 + np.arange(5), 64, CFG.dir_seed).numpy()
    np.testing.assert_allclose(d[..., :3], ref, atol=2e-6)
    assert np.all(d[..., 3] == 0)


@pytest.mark.parametrize("P, K", [(40, 64), (33, 36), (20, 169), (9, 400)])   # K > 128: several direction units per point
def test_distill_gradient_matches_oracle(lib, P, K):
    student, teacher = _scene(2), _scene(1)
    rs, rt = helpers.renderer_for(CFG, student), helpers.renderer_for(CFG, teacher)
    gb = scenegen.make_gbuffer(P, 4)
    pos = torch.from_numpy(gb["pos"]).cuda()
    nrm = torch.from_numpy(gb["normal"]).cuda()
    dirs = rs.distill_dirs(P, K)
    feat = rt.encode(pos)
    brdf_t = rt.decode(feat)
    vis_t, depth_t = rt.trace(feat, dirs)
    g_t = torch.zeros(student.table.size, device="cuda")
    g_b = torch.zeros(student.brdf_blob.size, device="cuda")
    g_i = torch.zeros(student.irt_blob.size, device="cuda")
    loss = torch.zeros(3, device="cuda")
    rs.distill_backward(pos, nrm, dirs, brdf_t, vis_t, depth_t, loss, g_t, g_b, g_i)
    torch.cuda.synchronize()
    assert rs.check() == 0

    # the oracle: its own directions, teacher targets (hit test in float32, as the teacher's stage kernel
    # takes it) and float64 gradient
    x = torch.from_numpy(gb["pos"][:, :3].astype(np.float64))
    n = torch.from_numpy(gb["normal"][:, :3].astype(np.float64))
    w = odist.stratified_sphere(np.arange(P), K, CFG.dir_seed)
    opt = orender.Options.from_config(CFG)
    prm_s = orender.Params.from_arrays(student.table, student.brdf, student.irt, student.env)
    prm_t = orender.Params.from_arrays(teacher.table, teacher.brdf, teacher.irt, teacher.env)
    tg = odist.teacher_targets(x, n, w, prm_t, opt, decision_arith="fp32")
    terms, r_t, r_b, r_i = odist.distill_gradient(x, n, w, prm_s, tg, opt)
    np.testing.assert_allclose(loss.cpu().numpy(), terms, rtol=2e-5)
    for got, ref in ((g_t, r_t), (g_b, r_b), (g_i, r_i)):
        got = got.cpu().numpy().reshape(-1).astype(np.float64)
        ref = ref.numpy().reshape(-1)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < 1e-4, rel


def test_adam_step_matches_oracle(lib):
    rng = np.random.default_rng(0)
    n = 1000
    p, g = rng.normal(size=n), rng.normal(size=n)
    m, v = rng.normal(size=n) * 0.1, rng.random(n) * 0.1
    t = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (p, g, m, v)]
    lib.adam_step(t[0], t[1], t[2], t[3], step=3, lr=0.01, weight_decay=1e-2)
    # the ABI takes float hyperparameters: the oracle gets the same float32 values (1 - beta2 is exact there)
    f = lambda a: float(np.float32(a))
    rp, rm, rv = odist.adam_step(p.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64),
                                 m.astype(np.float32).astype(np.float64), v.astype(np.float32).astype(np.float64),
                                 3, lr=f(0.01), beta1=f(0.9), beta2=f(0.999), eps=f(1e-8), weight_decay=f(1e-2))
    np.testing.assert_allclose(t[0].cpu().numpy(), rp, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(t[2].cpu().numpy(), rm, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(t[3].cpu().numpy(), rv, rtol=1e-5, atol=1e-9)


def test_training_lowers_the_loss(lib):
    from paper_2409_10327_gb300 import distill
    student, teacher = _scene(2), _scene(1)
    rs, rt = helpers.renderer_for(CFG, student), helpers.renderer_for(CFG, teacher)
    gb = scenegen.make_gbuffer(256, 6)
    pos = torch.from_numpy(gb["pos"]).cuda()
    nrm = torch.from_numpy(gb["normal"]).cuda()
    d = distill.Distiller(rs, rt, torch.from_numpy(student.table).cuda(), torch.from_numpy(student.brdf_blob).cuda(),
                          torch.from_numpy(student.irt_blob).cuda(), torch.from_numpy(student.env).cuda(), K=64)
    first = float(d.step(pos, nrm).sum())
    for _ in range(40):
        last = float(d.step(pos, nrm).sum())
    assert np.isfinite(last) and last < 0.7 * first, (first, last)


def test_bf16_student_is_rejected(lib):
    cfg = type(CFG)(**{**CFG.__dict__, "precision": "bf16"})
    sc = scenegen.make_scene(cfg, 2)
    r = helpers.renderer_for(cfg, sc)
    P, K = 4, 16
    z = lambda *s: torch.zeros(*s, device="cuda")
    with pytest.raises(lib.RtError) as e:
        r.distill_backward(z(P, 4), z(P, 4), z(P, K, 4), z(P, 8), z(P, K), z(P, K), None, z(sc.table.size),
                           z(sc.brdf_blob.size), z(sc.irt_blob.size))
    assert e.value.status == lib.RT_ERR_UNSUPPORTED
