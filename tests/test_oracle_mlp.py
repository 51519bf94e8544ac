"""Pins of the oracle's MLPs (stages (b), (c)) against numpy and closed forms."""
import math

import numpy as np
import pytest
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


# ---- the kernel arithmetic used for decisions (mlp3_arith) -------------------

def _one_path(w1, b1, w2, b2, w3, b3):
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    return [(t([[w1]]), t([b1])), (t([[w2]]), t([b2])), (t([[w3]]), t([b3]))]


@pytest.mark.parametrize("arith", ["bf16", "bf16x3", "fp32"])
def test_kernel_arith_is_exact_on_representable_values(arith):
    # one-hot layers with power-of-two weights and bf16-representable inputs: no rounding anywhere
    rng = np.random.default_rng(0)
    z = torch.tensor(rng.integers(-64, 64, (16, 8)) / 32.0, dtype=torch.float64)
    eye = lambda k, m, s: torch.tensor(np.eye(k, m) * s, dtype=torch.float64)
    layers = [(eye(8, 8, 0.5), torch.full((8,), 0.25, dtype=torch.float64)),
              (eye(8, 8, 2.0), torch.zeros(8, dtype=torch.float64)),
              (eye(3, 8, -1.0), torch.tensor([0.5, 0.0, -0.25], dtype=torch.float64))]
    np.testing.assert_array_equal(mlp.mlp3_arith(z, layers, arith).numpy(), mlp.mlp3(z, layers).numpy())


def test_bf16_arith_rounds_inputs_hidden_weights_and_activations_only():
    one = torch.tensor([[1.0]], dtype=torch.float64)
    # input 1 + 2^-9 is below half an ulp of bf16 at 1 (2^-8): rounds to 1
    z = torch.tensor([[1.0 + 2 ** -9]], dtype=torch.float64)
    assert mlp.mlp3_arith(z, _one_path(1, 0, 1, 0, 1, 0), "bf16").item() == 1.0
    assert mlp.mlp3(z, _one_path(1, 0, 1, 0, 1, 0)).item() == 1.0 + 2 ** -9
    # first hidden activation 1 + 2^-7 + 2^-9 rounds to 1 + 2^-7 (nearest bf16)
    h = mlp.mlp3_arith(one, _one_path(1 + 2 ** -7, 2 ** -9, 1, 0, 1, 0), "bf16").item()
    assert h == 1.0 + 2 ** -7
    # a hidden weight 1 + 2^-9 rounds to 1
    assert mlp.mlp3_arith(one, _one_path(1, 0, 1 + 2 ** -9, 0, 1, 0), "bf16").item() == 1.0
    # the second hidden activation and the output layer stay float32: 1 + 2^-20 survives
    assert mlp.mlp3_arith(one, _one_path(1, 0, 1, 2 ** -20, 1, 0), "bf16").item() == 1.0 + 2 ** -20
    assert mlp.mlp3_arith(one, _one_path(1, 0, 1, 0, 1 + 2 ** -20, 0), "bf16").item() == 1.0 + 2 ** -20
    # fp32 rounds 1 + 2^-30 away at every stage
    assert mlp.mlp3_arith(torch.tensor([[1.0 + 2 ** -30]], dtype=torch.float64),
                          _one_path(1, 0, 1, 0, 1, 0), "fp32").item() == 1.0


def test_bf16x3_arith_keeps_the_residual_and_drops_only_lo_times_lo():
    one = torch.tensor([[1.0]], dtype=torch.float64)
    # an input 1 + 2^-9 is 1 in bf16, but its residual 2^-9 survives the split product
    z = torch.tensor([[1.0 + 2 ** -9]], dtype=torch.float64)
    assert mlp.mlp3_arith(z, _one_path(1, 0, 1, 0, 1, 0), "bf16x3").item() == 1.0 + 2 ** -9
    # (1 + 2^-9)(1 + 2^-9) = 1 + 2^-8 + 2^-18: the split keeps hi.hi + lo.hi + hi.lo = 1 + 2^-8
    # (the hidden activation 1 + 2^-8 is itself split again for layer 2)
    assert mlp.mlp3_arith(z, _one_path(1 + 2 ** -9, 0, 1, 0, 1, 0), "bf16x3").item() == 1.0 + 2 ** -8
    assert mlp.mlp3(z, _one_path(1 + 2 ** -9, 0, 1, 0, 1, 0)).item() == 1.0 + 2 ** -8 + 2 ** -18
    # a hidden weight's residual survives too: 1 . (1 + 2^-9) = 1 + 2^-9 in layer 2
    assert mlp.mlp3_arith(one, _one_path(1, 0, 1 + 2 ** -9, 0, 1, 0), "bf16x3").item() == 1.0 + 2 ** -9
    # two bf16 parts hold about 16 significant bits: 1 + 2^-9 + 2^-17 keeps 1 + 2^-9
    z = torch.tensor([[1.0 + 2 ** -9 + 2 ** -17]], dtype=torch.float64)
    assert mlp.mlp3_arith(z, _one_path(1, 0, 1, 0, 1, 0), "bf16x3").item() == 1.0 + 2 ** -9
