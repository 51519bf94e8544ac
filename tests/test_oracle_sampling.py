"""Pins of the oracle's direction sampler: published RNG outputs and lobe statistics."""
import os

import numpy as np
import torch

from oracle import sampling

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")


def _golden():
    return [int(l, 16) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]


def test_splitmix64_published_outputs():
    got = sampling.splitmix64(0, np.arange(1, 4, dtype=np.uint64))
    assert [int(v) for v in got] == _golden()


def test_uniform24_is_exact_and_in_range():
    u = sampling.uniform24(sampling.splitmix64(123, np.arange(1, 10001, dtype=np.uint64)))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_counters_are_distinct():
    q = np.arange(0, 50, dtype=np.uint64)[:, None]
    slots = np.arange(0, 9, dtype=np.uint64)[None, :]
    c = sampling.counters(q, slots, 8)
    assert np.unique(c).size == c.size


def _normals(k, seed):
    n = np.random.default_rng(seed).normal(size=(k, 3))
    return torch.from_numpy(n / np.linalg.norm(n, axis=1, keepdims=True))


def test_uniform_sphere_moments():
    K = 400000
    u1, u2 = sampling.uniforms(7, np.arange(K, dtype=np.uint64))
    s = sampling.uniform_sphere(u1, u2)
    assert torch.allclose(s.norm(dim=1), torch.ones(K, dtype=torch.float64), atol=1e-12)
    se = 1.0 / np.sqrt(K)
    assert float(s.mean(0).abs().max()) < 5 * se
    cov = (s.T @ s / K).numpy()
    np.testing.assert_allclose(cov, np.eye(3) / 3, atol=5 * se)


def test_cosine_lobe_moments_and_support():
    K = 400000
    n = _normals(K, 3)
    u1, u2 = sampling.uniforms(11, np.arange(K, dtype=np.uint64))
    w = sampling.cosine_direction(n, u1, u2)
    assert torch.allclose(w.norm(dim=1), torch.ones(K, dtype=torch.float64), atol=1e-12)
    c = (w * n).sum(1)
    assert float(c.min()) >= -1e-12
    se = 1.0 / np.sqrt(K)
    # cos-weighted: pdf of mu = cos(theta) is 2 mu on [0, 1]
    assert abs(float(c.mean()) - 2.0 / 3.0) < 5 * se
    assert abs(float((c * c).mean()) - 0.5) < 5 * se
    # P(mu < 1/2) = 1/4
    assert abs(float((c < 0.5).double().mean()) - 0.25) < 5 * se


def test_cosine_lobe_azimuth_is_uniform_about_fixed_normal():
    K = 200000
    n = torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64).expand(K, 3)
    u1, u2 = sampling.uniforms(5, np.arange(K, dtype=np.uint64))
    w = sampling.cosine_direction(n, u1, u2)
    phi = torch.atan2(w[:, 1], w[:, 0])
    hist = np.histogram(phi.numpy(), bins=8, range=(-np.pi, np.pi))[0] / K
    np.testing.assert_allclose(hist, 1 / 8, atol=5 * np.sqrt(1 / 8 / K))
