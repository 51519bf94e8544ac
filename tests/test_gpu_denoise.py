"""rt_denoise (spatial SVGF, Sec. 4.1) against the oracle's float64 filter."""
import numpy as np
import pytest
import torch

from oracle import denoise as oden
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2409_10327_gb300 import build
    build.build()
    from paper_2409_10327_gb300 import binding
    return binding


def _image(h, w, seed=0):
    """Noisy radiance over a plane with incommensurate depth slopes, two depth steps and a normal edge."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    z = 2.0 + 0.013 * x + 0.0071 * y
    z[: h // 3, : w // 2] += 0.5                      # a raised patch
    z[h // 2:, w // 3:] -= 0.25
    n = np.zeros((h, w, 3))
    n[...] = [0.0, 0.28, 0.96]
    n[:, (2 * w) // 3:] = [0.6, 0.0, 0.8]             # a normal edge
    n += rng.normal(0, 0.02, n.shape)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    c = rng.lognormal(0.0, 0.7, (h, w, 3)) * (1.0 + 0.5 * (x[..., None] > w / 2))
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    return f32(c), f32(z), f32(n)


def _run(lib, c, z, n, **kw):
    h, w = z.shape
    pad = lambda a: np.concatenate([a.reshape(-1, 3), np.zeros((h * w, 1), np.float32)], 1)
    rad = torch.from_numpy(pad(c)).cuda()
    nrm = torch.from_numpy(pad(n)).cuda()
    dep = torch.from_numpy(z.reshape(-1)).cuda()
    out = lib.denoise(rad, dep, nrm, w, h, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(h, w, 4)


def _check(got, ref_c, ref_v):
    peak = float(np.abs(ref_c).max())
    err = np.abs(got[..., :3] - ref_c)
    assert float(err.max()) <= 1e-4 * peak, float(err.max() / peak)
    np.testing.assert_allclose(got[..., 3], ref_v, rtol=2e-3, atol=1e-6 * float(np.abs(ref_v).max() + 1e-30))


@pytest.mark.parametrize("h, w, iters", [(37, 45, 5), (20, 16, 3), (9, 50, 2)])
def test_denoise_matches_oracle(lib, h, w, iters):
    c, z, n = _image(h, w, h + w)
    got = _run(lib, c, z, n, iterations=iters)
    ref_c, ref_v = oden.svgf(c, z, n, iterations=iters)
    _check(got, ref_c, ref_v)


def test_zero_passes_return_the_variance_estimate(lib):
    c, z, n = _image(21, 19, 4)
    got = _run(lib, c, z, n, iterations=0)
    np.testing.assert_array_equal(got[..., :3], c)
    np.testing.assert_allclose(got[..., 3], oden.spatial_variance(c, z, n), rtol=2e-4, atol=1e-7)


@pytest.mark.parametrize("h, w", [(1, 1), (1, 7), (5, 1), (3, 3)])
def test_degenerate_sizes(lib, h, w):
    c, z, n = _image(max(h, 2), max(w, 2), 5)
    c, z, n = c[:h, :w].copy(), z[:h, :w].copy(), n[:h, :w].copy()
    got = _run(lib, c, z, n, iterations=4)
    ref_c, ref_v = oden.svgf(c, z, n, iterations=4)
    _check(got, ref_c, ref_v)


def test_constant_image_is_unchanged(lib):
    c, z, n = _image(24, 24, 6)
    c[:] = np.array([0.25, 1.5, 3.0], np.float32)
    got = _run(lib, c, z, n)
    np.testing.assert_allclose(got[..., :3], c, rtol=1e-6)


def test_denoise_argument_errors(lib):
    P = 16
    t = lambda: torch.zeros(P, 4, device="cuda")
    rad, nrm, work, out = t(), t(), t(), t()
    dep = torch.zeros(P, device="cuda")
    call = lambda **kw: lib.LIB.rt_denoise(kw.get("w", 4), kw.get("h", 4), lib._ptr(kw.get("rad", rad)),
                                           lib._ptr(dep), lib._ptr(nrm), kw.get("it", 5), kw.get("sz", 1.0), 128.0,
                                           4.0, lib._ptr(kw.get("work", work)), lib._ptr(kw.get("out", out)), None)
    assert call() == lib.RT_OK
    assert call(it=13) == lib.RT_ERR_INVALID_ARG
    assert call(w=0) == lib.RT_ERR_INVALID_ARG
    assert call(sz=0.0) == lib.RT_ERR_INVALID_ARG
    assert call(out=rad) == lib.RT_ERR_INVALID_ARG          # output over the input
    assert call(work=out) == lib.RT_ERR_INVALID_ARG
    torch.cuda.synchronize()


def test_denoised_render(lib):
    # the rendered 64 x 64 frame, depth = distance to a camera at (0, 0, -3): same filter on both sides
    import scenegen
    cfg = scenegen.CONFIGS["tiny64"]
    sc, gb = helpers.scene_arrays(cfg, 0)
    r = helpers.renderer_for(cfg, sc)
    dgb = helpers.to_cuda(gb)
    rad = r.render_frame(dgb)
    pos = gb["pos"][:, :3].astype(np.float64)
    z = np.linalg.norm(pos - np.array([0.0, 0.0, -3.0]), axis=1).astype(np.float32)
    out = lib.denoise(rad, torch.from_numpy(z).cuda(), dgb["normal"], 64, 64, iterations=3).cpu().numpy()
    c = rad.cpu().numpy()[:, :3].reshape(64, 64, 3)
    ref_c, ref_v = oden.svgf(c, z.reshape(64, 64), gb["normal"][:, :3].reshape(64, 64, 3), iterations=3)
    _check(out.reshape(64, 64, 4), ref_c, ref_v)
