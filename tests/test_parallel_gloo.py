"""The N-rank path on CPU: world size 2 over gloo (127.0.0.1)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import scenegen
from oracle import distill as odist
from oracle import render as orender
from paper_2409_10327_gb300 import parallel

CFG = scenegen.SceneConfig("g", 6, 5, 8, m_dirs=2, levels=4, log2_T=10, base_res=4, max_res=32, env_h=8, env_w=16)
DCFG = scenegen.SceneConfig("d", 8, 1, 16, levels=4, log2_T=10, base_res=4, max_res=32)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # 1. a frame rendered in pixel shards (pixel_offset keys the RNG) and gathered
        sc = scenegen.make_scene(CFG, 0, bias_scale=0.1)
        gb = scenegen.make_gbuffer(CFG.n_pixels, 0)
        prm = orender.Params.from_arrays(sc.table, sc.brdf, sc.irt, sc.env)
        opt = orender.Options.from_config(CFG)
        lo, hi = parallel.shard_range(CFG.n_pixels, world, rank)
        part = orender.render({k: v[lo:hi] for k, v in gb.items()}, prm, opt, pixel_offset=lo)
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, part))
        # 2. timing reduction
        mx = parallel.max_over_ranks(float(rank + 1) * 2.5)
        # 3. data-parallel distillation gradient: each rank takes half the rays
        st = orender.Params.from_arrays(*[getattr(scenegen.make_scene(DCFG, 2, bias_scale=0.1), a)
                                          for a in ("table", "brdf", "irt", "env")])
        te = orender.Params.from_arrays(*[getattr(scenegen.make_scene(DCFG, 1, bias_scale=0.1), a)
                                          for a in ("table", "brdf", "irt", "env")])
        dgb = scenegen.make_gbuffer(DCFG.n_pixels, 3)
        r0, r1 = parallel.shard_range(DCFG.n_pixels, world, rank)
        x = torch.from_numpy(dgb["pos"][r0:r1, :3].astype(np.float64))
        n = torch.from_numpy(dgb["normal"][r0:r1, :3].astype(np.float64))
        w = odist.stratified_sphere(np.arange(r0, r1), 16, DCFG.dir_seed)
        dopt = orender.Options.from_config(DCFG)
        tg = odist.teacher_targets(x, n, w, te, dopt)
        _, gt, gbr, gi = odist.distill_gradient(x, n, w, st, tg, dopt)
        grads = [gt.clone(), gbr.clone(), gi.clone()]
        parallel.allreduce_mean(grads)
        if rank == 0:
            torch.save({"parts": parts, "max": mx, "grads": grads}, os.path.join(out_dir, "rank0.pt"))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = torch.load(os.path.join(tmp_path, "rank0.pt"), weights_only=False)
    # shards cover the frame, and the gathered frame equals the whole frame exactly
    sc = scenegen.make_scene(CFG, 0, bias_scale=0.1)
    gb = scenegen.make_gbuffer(CFG.n_pixels, 0)
    prm = orender.Params.from_arrays(sc.table, sc.brdf, sc.irt, sc.env)
    whole = orender.render(gb, prm, orender.Options.from_config(CFG))
    spans = sorted((lo, hi) for lo, hi, _ in res["parts"])
    assert spans[0][0] == 0 and spans[-1][1] == CFG.n_pixels and spans[0][1] == spans[1][0]
    gathered = np.concatenate([p for _, _, p in sorted(res["parts"], key=lambda t: t[0])])
    np.testing.assert_array_equal(gathered, whole)
    assert res["max"] == 5.0
    # the averaged half-batch gradients are the full batch's gradient
    st = orender.Params.from_arrays(*[getattr(scenegen.make_scene(DCFG, 2, bias_scale=0.1), a)
                                      for a in ("table", "brdf", "irt", "env")])
    te = orender.Params.from_arrays(*[getattr(scenegen.make_scene(DCFG, 1, bias_scale=0.1), a)
                                      for a in ("table", "brdf", "irt", "env")])
    dgb = scenegen.make_gbuffer(DCFG.n_pixels, 3)
    x = torch.from_numpy(dgb["pos"][:, :3].astype(np.float64))
    n = torch.from_numpy(dgb["normal"][:, :3].astype(np.float64))
    w = odist.stratified_sphere(np.arange(DCFG.n_pixels), 16, DCFG.dir_seed)
    dopt = orender.Options.from_config(DCFG)
    _, gt, gbr, gi = odist.distill_gradient(x, n, w, st, odist.teacher_targets(x, n, w, te, dopt), dopt)
    for got, ref in zip(res["grads"], (gt, gbr, gi)):
        np.testing.assert_allclose(got.numpy(), ref.numpy(), rtol=1e-10, atol=1e-14)


def test_shard_ranges():
    for n in (0, 1, 7, 640000):
        for world in (1, 2, 3, 8):
            spans = [parallel.shard_range(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1
    with pytest.raises(ValueError):
        parallel.shard_range(5, 2, 2)
