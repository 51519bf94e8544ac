"""Pins of the oracle's hash-grid encoder (stage (a)) against closed forms and brute force."""
import itertools

import numpy as np
import pytest
import torch

from oracle import hashgrid


def test_paper_resolution_ladder_is_powers_of_two():
    # Sec. 4.1: 14 levels from 16 to 131072 -> growth factor b = 2 exactly.
    res = hashgrid.level_resolutions(14, 16, 131072)
    assert res == [16 * 2 ** l for l in range(14)]


@pytest.mark.parametrize("levels,nmin,nmax", [(16, 16, 2048), (8, 16, 256), (4, 3, 40)])
def test_resolution_ladder_properties(levels, nmin, nmax):
    res = hashgrid.level_resolutions(levels, nmin, nmax)
    assert res[0] == nmin and res[-1] == nmax
    b = (nmax / nmin) ** (1.0 / (levels - 1))
    for l, r in enumerate(res):
        exact = nmin * b ** l
        assert r <= exact + 1e-6 and r > exact - 1.0


def test_dense_index_is_a_bijection():
    res, T = 5, 1 << 10
    ijk = torch.tensor(list(itertools.product(range(res + 1), repeat=3)))
    idx = hashgrid.corner_index(ijk[:, 0], ijk[:, 1], ijk[:, 2], res, T, True)
    assert sorted(idx.tolist()) == list(range((res + 1) ** 3))
    # x is the fastest axis, then y (stride N+1), then z (stride (N+1)^2)
    one = torch.tensor([1])
    zero = torch.tensor([0])
    assert hashgrid.corner_index(one, zero, zero, res, T, True).item() == 1
    assert hashgrid.corner_index(zero, one, zero, res, T, True).item() == res + 1
    assert hashgrid.corner_index(zero, zero, one, res, T, True).item() == (res + 1) ** 2


def test_hash_axes_and_xor_separability():
    T32 = 1 << 32
    one, zero = torch.tensor([1]), torch.tensor([0])
    # With T = 2^32 a unit step along each axis returns that axis' prime (Instant-NGP).
    assert hashgrid.corner_index(one, zero, zero, 7, T32, False).item() == 1
    assert hashgrid.corner_index(zero, one, zero, 7, T32, False).item() == 2654435761
    assert hashgrid.corner_index(zero, zero, one, 7, T32, False).item() == 805459861
    rng = np.random.default_rng(0)
    T = 1 << 14
    i, j, k = (torch.from_numpy(rng.integers(0, 3000, 500)) for _ in range(3))
    z = torch.zeros_like(i)
    full = hashgrid.corner_index(i, j, k, 2999, T, False)
    sep = (hashgrid.corner_index(i, z, z, 2999, T, False) ^ hashgrid.corner_index(z, j, z, 2999, T, False)
           ^ hashgrid.corner_index(z, z, k, 2999, T, False))
    assert torch.equal(full, sep)
    assert int(full.min()) >= 0 and int(full.max()) < T
    # the x prime is 1: along x alone the hash is the coordinate mod T
    assert torch.equal(hashgrid.corner_index(i, z, z, 2999, T, False), i % T)


def _table(L, T, F, seed=0):
    return torch.from_numpy(np.random.default_rng(seed).uniform(-0.1, 0.1, (L, T, F)))


def test_weights_sum_to_one_and_range():
    res = hashgrid.level_resolutions(8, 16, 256)
    dense = hashgrid.dense_levels(res, 1 << 14)
    x = torch.from_numpy(np.random.default_rng(1).uniform(-1.4, 1.4, (2000, 3)))
    _, idx, w = hashgrid.encode(x, _table(8, 1 << 14, 2), res, dense, return_aux=True)
    assert torch.allclose(w.sum(-1), torch.ones(2000, 8, dtype=torch.float64), atol=1e-14)
    assert float(w.min()) >= 0.0
    assert int(idx.min()) >= 0 and int(idx.max()) < (1 << 14)


@pytest.mark.parametrize("fp32_grid", [False, True])
def test_lattice_vertices_return_table_entries(fp32_grid):
    # Dyadic resolutions (b = 2): x = 2 v / N_l - 1 is exact, so g = v exactly.
    res = [4, 8, 16, 32]
    T = 1 << 10
    dense = hashgrid.dense_levels(res, T)
    assert dense == [True, True, False, False]
    table = _table(4, T, 2, 3)
    rng = np.random.default_rng(2)
    for l, r in enumerate(res):
        v = rng.integers(0, r + 1, (64, 3))
        x = torch.from_numpy(2.0 * v / r - 1.0)
        f = hashgrid.encode(x, table, res, dense, fp32_grid=fp32_grid)
        vt = torch.from_numpy(v)
        rows = hashgrid.corner_index(vt[:, 0], vt[:, 1], vt[:, 2], r, T, dense[l])
        assert torch.equal(f[:, 2 * l:2 * l + 2], table[l][rows])


def test_brute_force_tent_functions_on_tiny_grids():
    # f_l(x) = sum over ALL vertices v of prod_d max(0, 1 - |g_d - v_d|) * table[idx(v)]
    # (no floor, no cell): covers dense and hashed levels, boundary and clamped points.
    res = [2, 3, 4]
    T = 64
    dense = hashgrid.dense_levels(res, T)
    assert dense == [True, True, False]
    table = _table(3, T, 2, 4)
    rng = np.random.default_rng(5)
    pts = np.concatenate([rng.uniform(-1.2, 1.2, (40, 3)), np.array([[1.0, -1.0, 1.0], [0.0, 0.5, -0.25]])])
    f = hashgrid.encode(torch.from_numpy(pts), table, res, dense)
    for p, x in enumerate(pts):
        for l, r in enumerate(res):
            g = np.clip((x + 1.0) / 2.0, 0.0, 1.0) * r
            acc = np.zeros(2)
            for v in itertools.product(range(r + 1), repeat=3):
                wt = np.prod([max(0.0, 1.0 - abs(g[d] - v[d])) for d in range(3)])
                if wt == 0.0:
                    continue
                row = hashgrid.corner_index(torch.tensor(v[0]), torch.tensor(v[1]), torch.tensor(v[2]),
                                            r, T, dense[l]).item()
                acc += wt * table[l, row].numpy()
            np.testing.assert_allclose(f[p, 2 * l:2 * l + 2].numpy(), acc, rtol=0, atol=1e-15)


def test_fp32_grid_matches_fp64_grid_away_from_cell_faces():
    res = hashgrid.level_resolutions(16, 16, 2048)
    dense = hashgrid.dense_levels(res, 1 << 19)
    x32 = np.random.default_rng(6).uniform(-1, 1, (4000, 3)).astype(np.float32)
    x = torch.from_numpy(x32.astype(np.float64))
    table = _table(16, 1 << 19, 2, 7)
    f64, i64, w64 = hashgrid.encode(x, table, res, dense, return_aux=True)
    f32, i32, w32 = hashgrid.encode(x, table, res, dense, fp32_grid=True, return_aux=True)
    same = (i64 == i32).all(-1)
    assert float(same.double().mean()) > 0.999
    # where the cells agree, w differs by the float32 roundings of u (2^-24 near 1,
    # times N_l) and of g = u N_l (half an ulp of a number below 2 N_l)
    for l, r in enumerate(res):
        ok = same[:, l]
        assert float((w64[ok, l] - w32[ok, l]).abs().max()) <= 3 * 2.0 * r * 2.0 ** -24 + 1e-12
