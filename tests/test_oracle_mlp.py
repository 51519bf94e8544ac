"""Pins of the oracle's MLPs (stages (b), (c)) against numpy and closed forms."""
import math

import numpy as np
import torch

import scenegen
from oracle import mlp


def _np_mlp(z, layers):
    h = z
    for k, (w, b) in enumerate(layers):
        h = h @ np.asarray(w, np.float64).T + np.asarray(b, np.float64)
        if k < 2:
            h = np.maximum(h, 0.0)
    return h


def test_mlp3_matches_numpy_chain():
    layers = scenegen.make_mlp(59, 2, seed=3, stream=11, bias_scale=0.2)
    z = np.random.default_rng(0).normal(size=(300, 59))
    got = mlp.mlp3(torch.from_numpy(z), mlp.as_layers(layers)).numpy()
    np.testing.assert_allclose(got, _np_mlp(z, layers), rtol=1e-13, atol=1e-14)


def test_brdf_decoder_closed_form_from_output_bias():
    # Zero weights: the output equals b3, so n, a, r follow from b3 alone.
    layers = [(np.zeros((64, 32)), np.zeros(64)), (np.zeros((64, 64)), np.zeros(64)),
              (np.zeros((7, 64)), np.array([3.0, 0.0, -4.0, 0.0, 1.0, -2.0, 0.5]))]
    a, r, n = mlp.brdf_decoder(torch.zeros(3, 32, dtype=torch.float64), mlp.as_layers(layers))
    np.testing.assert_allclose(n[0].numpy(), [0.6, 0.0, -0.8], atol=1e-15)
    sig = lambda t: 1.0 / (1.0 + math.exp(-t))
    np.testing.assert_allclose(a[0].numpy(), [0.5, sig(1.0), sig(-2.0)], atol=1e-15)
    assert abs(float(r[0]) - (0.09 + 0.91 * sig(0.5))) < 1e-15


def test_brdf_decoder_ranges():
    layers = mlp.as_layers(scenegen.make_mlp(32, 7, seed=1, stream=10, bias_scale=1.0))
    f = torch.from_numpy(np.random.default_rng(1).normal(size=(500, 32)))
    a, r, n = mlp.brdf_decoder(f, layers)
    assert torch.allclose(n.norm(dim=1), torch.ones(500, dtype=torch.float64), atol=1e-14)
    assert float(a.min()) > 0 and float(a.max()) < 1
    assert float(r.min()) > 0.09 and float(r.max()) < 1.0


def test_positional_encoding_closed_forms():
    pe = mlp.positional_encoding(torch.tensor([[0.0, 0.0, 0.0], [1.0, 0.0, -0.5]], dtype=torch.float64))
    assert pe.shape == (2, 27)
    np.testing.assert_allclose(pe[0].numpy(), [0, 0, 0] + ([0, 0, 0] + [1, 1, 1]) * 4, atol=1e-15)
    # w = (1, 0, -1/2): sin(2^k pi) = 0, cos(2^k pi) = (-1)^[k==0]; sin(-pi/2)=-1, cos(-pi/2)=0, ...
    want = [1.0, 0.0, -0.5,
            0.0, 0.0, -1.0, -1.0, 1.0, 0.0,        # k=0: sin(pi w), cos(pi w)
            0.0, 0.0, 0.0, 1.0, 1.0, -1.0,         # k=1: sin(2 pi w), cos(2 pi w)
            0.0, 0.0, 0.0, 1.0, 1.0, 1.0,          # k=2
            0.0, 0.0, 0.0, 1.0, 1.0, 1.0]          # k=3
    np.testing.assert_allclose(pe[1].numpy(), want, atol=1e-14)


def test_irt_outputs_and_depth_mapping():
    near, far = 0.05, 1.5
    zero = [(np.zeros((64, 59)), np.zeros(64)), (np.zeros((64, 64)), np.zeros(64)),
            (np.zeros((2, 64)), np.zeros(2))]
    f = torch.zeros(4, 32, dtype=torch.float64)
    w = torch.tensor([[0.0, 0.0, 1.0]] * 4, dtype=torch.float64)
    v, t = mlp.implicit_ray_tracer(f, w, mlp.as_layers(zero), near, far)
    assert torch.allclose(v, torch.full((4,), 0.5, dtype=torch.float64))
    assert torch.allclose(t, torch.full((4,), near + (far - near) * math.log(2.0), dtype=torch.float64))
    assert float(mlp.depth_from_logit(torch.tensor(0.0, dtype=torch.float64), near, far)) == near
    assert float(mlp.depth_from_logit(torch.tensor(7.0, dtype=torch.float64), near, far)) == far
