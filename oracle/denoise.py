"""Spatial SVGF denoiser applied to the raw Monte Carlo frame  (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper denoises its renders with SVGF (Schied et al. 2017) with every
temporal element removed (Sec. 4.1), and takes the depth gradient from the
depth map offset by one pixel horizontally and vertically (supplementary
"Rendering Details").  What remains, per pixel p of a W x H image with
colour c, unit normal n, depth z and luminance l = 0.2126 R + 0.7152 G +
0.0722 B:

1. Variance estimate.  With no history SVGF estimates the luminance
   variance spatially: over the 7 x 7 window around p, with weights
   w = w_z w_n (below, step 1),  Var(p) = max(0, E[l^2] - E[l]^2) of the
   weighted moments.
2. `iterations` a-trous passes with step s = 2^i: over the 5 x 5 taps
   q = p + s (dx, dy), dx, dy in -2..2,
      w(p, q) = h(dx) h(dy) w_z w_n w_l,   h = [1, 4, 6, 4, 1] / 16 (B3 spline)
      w_z = exp(-|z(p) - z(q)| / (sigma_z |grad z(p) . s (dx, dy)| + eps))
      w_n = max(0, n(p) . n(q)) ^ sigma_n
      w_l = exp(-|l(p) - l(q)| / (sigma_l sqrt(g(p)) + eps))
   with g the 3 x 3 Gaussian ([1, 2, 1] x [1, 2, 1] / 16) of the variance,
   then  c'(p) = sum w c(q) / sum w  and  Var'(p) = sum w^2 Var(q) / (sum w)^2.
   grad z(p) = (z(x+1, y) - z(x, y), z(x, y+1) - z(x, y)), backward at the
   last column and row.  Taps outside the image are skipped and sums are
   normalised by the weights that remain.

Readings: sigma_z = 1, sigma_n = 128, sigma_l = 4 and 5 passes are SVGF's
published defaults; eps = 1e-10; the spatial variance estimate uses depth and
normal weights only (SVGF names those two for it).

Pins (tests/test_oracle_denoise.py): a constant image is unchanged; with the
edge-stopping terms switched off the passes equal the composed dilated
B3-spline convolution (scipy) away from the border; a normal edge stops
all bleeding; the unweighted variance equals the window's plain variance;
one unweighted pass scales a constant variance by (70/256)^2.
"""
from __future__ import annotations

import numpy as np

H1 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0
EPS = 1e-10
LUMA = np.array([0.2126, 0.7152, 0.0722])


def depth_gradient(z: np.ndarray) -> np.ndarray:
    """[H, W, 2]: forward differences along x and y, backward at the last column / row."""
    gx = np.empty_like(z)
    gy = np.empty_like(z)
    gx[:, :-1] = z[:, 1:] - z[:, :-1]
    gx[:, -1] = z[:, -1] - z[:, -2] if z.shape[1] > 1 else 0.0
    gy[:-1, :] = z[1:, :] - z[:-1, :]
    gy[-1, :] = z[-1, :] - z[-2, :] if z.shape[0] > 1 else 0.0
    return np.stack([gx, gy], axis=-1)


def _w_geom(p, q, z, n, grad, step_xy, sigma_z, sigma_n):
    """Depth and normal edge-stopping weights between pixel p and pixel q (index tuples)."""
    dz = abs(z[p] - z[q])
    wz = np.exp(-dz / (sigma_z * abs(grad[p][0] * step_xy[0] + grad[p][1] * step_xy[1]) + EPS))
    wn = max(0.0, float(np.dot(n[p], n[q]))) ** sigma_n
    return wz * wn


def spatial_variance(c, z, n, sigma_z=1.0, sigma_n=128.0):
    """Var [H, W] from the 7 x 7 depth/normal-weighted luminance moments."""
    Hh, W = z.shape
    lum = c @ LUMA
    grad = depth_gradient(z)
    var = np.zeros((Hh, W))
    for y in range(Hh):
        for x in range(W):
            s0 = s1 = s2 = 0.0
            for dy in range(-3, 4):
                for dx in range(-3, 4):
                    qy, qx = y + dy, x + dx
                    if not (0 <= qy < Hh and 0 <= qx < W):
                        continue
                    w = _w_geom((y, x), (qy, qx), z, n, grad, (dx, dy), sigma_z, sigma_n)
                    s0 += w
                    s1 += w * lum[qy, qx]
                    s2 += w * lum[qy, qx] ** 2
            m1, m2 = s1 / s0, s2 / s0
            var[y, x] = max(0.0, m2 - m1 * m1)
    return var


def gaussian3(v):
    """3 x 3 Gaussian ([1, 2, 1] x [1, 2, 1] / 16) with out-of-image taps skipped and renormalised."""
    Hh, W = v.shape
    k = np.array([1.0, 2.0, 1.0])
    out = np.zeros_like(v)
    for y in range(Hh):
        for x in range(W):
            s = ws = 0.0
            for dy in range(-1, 2):
                for dx in range(-1, 2):
                    qy, qx = y + dy, x + dx
                    if 0 <= qy < Hh and 0 <= qx < W:
                        w = k[dy + 1] * k[dx + 1]
                        s += w * v[qy, qx]
                        ws += w
            out[y, x] = s / ws
    return out


def atrous_pass(c, var, z, n, step, sigma_z=1.0, sigma_n=128.0, sigma_l=4.0):
    """One a-trous pass with step `step`: (c' [H, W, 3], Var' [H, W])."""
    Hh, W = z.shape
    lum = c @ LUMA
    grad = depth_gradient(z)
    g = gaussian3(var)
    c2 = np.zeros_like(c)
    v2 = np.zeros_like(var)
    for y in range(Hh):
        for x in range(W):
            ws = 0.0
            acc = np.zeros(3)
            accv = 0.0
            den_l = sigma_l * np.sqrt(max(g[y, x], 0.0)) + EPS
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    qy, qx = y + step * dy, x + step * dx
                    if not (0 <= qy < Hh and 0 <= qx < W):
                        continue
                    w = H1[dy + 2] * H1[dx + 2]
                    w *= _w_geom((y, x), (qy, qx), z, n, grad, (step * dx, step * dy), sigma_z, sigma_n)
                    w *= np.exp(-abs(lum[y, x] - lum[qy, qx]) / den_l)
                    ws += w
                    acc += w * c[qy, qx]
                    accv += w * w * var[qy, qx]
            c2[y, x] = acc / ws
            v2[y, x] = accv / (ws * ws)
    return c2, v2


def svgf(c, z, n, iterations=5, sigma_z=1.0, sigma_n=128.0, sigma_l=4.0):
    """Denoised colour [H, W, 3] and the final variance [H, W] (all float64)."""
    c = np.asarray(c, np.float64)
    z = np.asarray(z, np.float64)
    n = np.asarray(n, np.float64)
    var = spatial_variance(c, z, n, sigma_z, sigma_n)
    for i in range(iterations):
        c, var = atrous_pass(c, var, z, n, 1 << i, sigma_z, sigma_n, sigma_l)
    return c, var
