"""Pins of the oracle's spatial SVGF denoiser."""
import numpy as np
import pytest

from oracle import denoise


def _scene(h=24, w=20, seed=0):
    rng = np.random.default_rng(seed)
    c = rng.lognormal(0.0, 1.0, (h, w, 3))
    z = 2.0 + np.cumsum(rng.normal(0, 0.01, (h, w)), axis=1)
    n = rng.normal(0, 1, (h, w, 3))
    n[..., 2] = np.abs(n[..., 2]) + 4.0
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    return c, z, n


def test_constant_image_is_unchanged():
    c, z, n = _scene()
    c[:] = np.array([0.3, 1.5, 2.0])
    out, var = denoise.svgf(c, z, n, iterations=3)
    np.testing.assert_allclose(out, c, rtol=1e-12)
    assert np.all(var <= 1e-12)   # E[l^2] - E[l]^2 of a constant, up to rounding


def test_without_edge_stopping_equals_the_composed_b3_convolution():
    scipy_ndimage = pytest.importorskip("scipy.ndimage")
    # flat constant depth and one normal make w_z = w_n = 1; a huge sigma_l makes w_l = 1
    h = w = 40
    c, z, n = _scene(h, w, 1)
    z[:] = 2.0
    n[:] = [0.0, 0.6, 0.8]
    out, _ = denoise.svgf(c, z, n, iterations=2, sigma_l=1e300)
    ref = c.copy()
    for i in range(2):
        s = 1 << i
        k = np.zeros((4 * s + 1, 4 * s + 1))
        k[::s, ::s] = np.outer(denoise.H1, denoise.H1)
        ref = np.stack([scipy_ndimage.convolve(ref[..., ch], k, mode="constant") for ch in range(3)], -1)
    m = 2 * (1 + 2)   # taps reach 2 (1 + 2) pixels: compare where no tap left the image
    np.testing.assert_allclose(out[m:-m, m:-m], ref[m:-m, m:-m], rtol=1e-12)


def test_a_normal_edge_stops_all_bleeding():
    h, w = 16, 16
    c = np.zeros((h, w, 3))
    c[:, : w // 2] = [1.0, 0.5, 0.25]
    c[:, w // 2:] = [4.0, 2.0, 8.0]
    z = np.full((h, w), 3.0)
    n = np.zeros((h, w, 3))
    n[:, : w // 2] = [0.0, 0.0, 1.0]
    n[:, w // 2:] = [1.0, 0.0, 0.0]
    out, _ = denoise.svgf(c, z, n, iterations=4)
    np.testing.assert_allclose(out, c, rtol=1e-12)


def test_unweighted_variance_is_the_window_variance():
    c, z, n = _scene(12, 12, 2)
    z[:] = 1.5
    n[:] = [0.0, 0.0, 1.0]
    var = denoise.spatial_variance(c, z, n)
    lum = c @ denoise.LUMA
    y, x = 6, 5
    win = lum[y - 3:y + 4, x - 3:x + 4]
    assert var[y, x] == pytest.approx(win.var(), rel=1e-12)


def test_one_unweighted_pass_scales_a_constant_variance():
    c, z, n = _scene(12, 12, 3)
    c[:] = 1.0
    z[:] = 1.5
    n[:] = [0.0, 0.0, 1.0]
    var = np.full(z.shape, 0.5)
    _, v2 = denoise.atrous_pass(c, var, z, n, 1)
    assert v2[6, 6] == pytest.approx(0.5 * (70.0 / 256.0) ** 2, rel=1e-12)
