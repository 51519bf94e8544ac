"""Stage (a): multi-resolution hash-grid encoding f = H(x)  (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper builds H "with multi-level tables as InstantNGP" (Sec. 3.2,
"Indirect Illumination Renderer") and gives its sizes in Sec. 4.1 (14
levels, T = 2^17, F = 2, resolutions 16 -> 131072).  The encoding is
therefore Instant-NGP's published one:

  * level l has resolution N_l = floor(N_min * b^l), b = exp((ln N_max -
    ln N_min) / (L - 1));
  * a point is mapped to grid coordinates g = u * N_l, u = (x + 1) / 2 for
    the domain [-1, 1]^3, clamped to [0, 1] (reading: the paper is silent
    on points outside the box; secondary points x' can leave it);
  * the 8 corners of the enclosing cell are looked up, densely (i + j(N+1)
    + k(N+1)^2) where (N_l+1)^3 <= T, else through the spatial hash
    (i*1 XOR j*2654435761 XOR k*805459861) mod T;
  * the corner features are blended with trilinear weights and the levels
    are concatenated level-major, F inner.

Pins (tests/test_oracle_hashgrid.py): weights sum to 1; lattice vertices
return table entries exactly; brute-force tent-function enumeration over
all vertices of tiny grids; closed forms of the hash on the axes and its
XOR separability; the paper's b = 2 resolution ladder.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import torch

# Instant-NGP's spatial-hash primes, one per axis (x, y, z).
HASH_PRIMES = (1, 2654435761, 805459861)


def level_resolutions(levels: int, base_res: int, max_res: int) -> List[int]:
    """N_l = floor(N_min * b^l) with the geometric growth factor b.

    A 1e-9 guard keeps exact integers such as N_max itself from being
    floored one below by the rounding of exp/log.
    """
    if levels == 1:
        return [int(base_res)]
    b = math.exp((math.log(max_res) - math.log(base_res)) / (levels - 1))
    return [int(math.floor(base_res * b ** l + 1e-9)) for l in range(levels)]


def dense_levels(res: Sequence[int], table_size: int, dense_coarse: bool = True) -> List[bool]:
    """A level is stored densely (1:1) when its (N_l+1)^3 vertices fit in T."""
    return [bool(dense_coarse) and (r + 1) ** 3 <= table_size for r in res]


def corner_index(ix: torch.Tensor, iy: torch.Tensor, iz: torch.Tensor,
                 res: int, table_size: int, dense: bool) -> torch.Tensor:
    """Table row of lattice vertex (ix, iy, iz) on a level of resolution res."""
    if dense:
        n1 = res + 1
        return ix + iy * n1 + iz * n1 * n1
    h = (ix * HASH_PRIMES[0]) ^ (iy * HASH_PRIMES[1]) ^ (iz * HASH_PRIMES[2])
    # (h mod 2^32) mod T == h mod T because T is a power of two <= 2^32.
    return h & (table_size - 1)


def grid_coords(x: torch.Tensor, res: int, fp32_grid: bool) -> Tuple[torch.Tensor, torch.Tensor]:
    """Cell origin i0 (int64) and fractional position w in [0, 1] (float64).

    fp32_grid=False: u and g = u * N_l in float64 (the render oracle).
    fp32_grid=True : u = x*0.5 + 0.5 and g = u * N_l rounded to IEEE float32,
    op by op, so that the integer cell decision is taken in the same
    precision as the float32 kernel (the cell index is an integer decided by
    floating point).  w = g - i0 is then exact in both precisions.
    """
    if fp32_grid:
        u = x.to(torch.float32) * 0.5 + 0.5
        u = u.clamp(0.0, 1.0)
        g32 = u * float(res)
        i0 = torch.floor(g32).to(torch.int64).clamp(max=res - 1)
        w = g32.to(torch.float64) - i0.to(torch.float64)
        return i0, w
    u = (x * 0.5 + 0.5).clamp(0.0, 1.0)
    g = u * float(res)
    i0 = torch.floor(g.detach()).to(torch.int64).clamp(max=res - 1)
    return i0, g - i0.to(g.dtype)


def encode(x: torch.Tensor, table: torch.Tensor, res: Sequence[int], dense: Sequence[bool],
           fp32_grid: bool = False, return_aux: bool = False):
    """f = H(x): concatenated trilinearly interpolated features of all levels.

    x      [P, 3]
    table  [L, T, F] float64
    returns f [P, L*F] (float64); with return_aux also the corner rows
    idx [P, L, 8] (int64) and weights w [P, L, 8] (float64), corner c having
    offsets (c & 1, (c >> 1) & 1, (c >> 2) & 1) along (x, y, z).
    """
    n_levels, table_size, feat = table.shape
    assert n_levels == len(res)
    feats, idxs, wts = [], [], []
    for l, r in enumerate(res):
        i0, w = grid_coords(x, r, fp32_grid)
        f_l = torch.zeros(x.shape[0], feat, dtype=torch.float64)
        li, lw = [], []
        for c in range(8):
            off = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
            idx = corner_index(i0[:, 0] + off[0], i0[:, 1] + off[1], i0[:, 2] + off[2],
                               r, table_size, dense[l])
            wt = torch.ones(x.shape[0], dtype=torch.float64)
            for d in range(3):
                wt = wt * (w[:, d] if off[d] else 1.0 - w[:, d])
            f_l = f_l + wt[:, None] * table[l][idx]
            li.append(idx)
            lw.append(wt)
        feats.append(f_l)
        idxs.append(torch.stack(li, dim=1))
        wts.append(torch.stack(lw, dim=1))
    f = torch.cat(feats, dim=1)
    if return_aux:
        return f, torch.stack(idxs, dim=1), torch.stack(wts, dim=1)
    return f
