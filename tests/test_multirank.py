"""Sharding across ranks without a GPU: two gloo ranks each render a disjoint
contiguous source range (global source indices), all-reduce the int64
fixed-point images, and must reproduce the single-process image bit for
bit; the same ranks split the dots of the Sec. 4 BOS experiment and gather
the per-dot displacements.  The oracle computes the partial results here
(CPU ranks)."""
import os
import socket

import numpy as np
import pytest

from paper_1812_05902_gb300 import scenes
from paper_1812_05902_gb300.shard import source_range


def test_source_ranges_cover_and_balance():
    for n in (1, 2, 7, 100, 4097):
        for world in (1, 2, 3, 8):
            spans = [source_range(n, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (f0, c0), (f1, c1) in zip(spans, spans[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in spans) == n
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        source_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1812_05902_gb300.shard import allreduce_image
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fr = scenes.c0(scale=0.05, rays_per_source=30)[0]
    first, count = source_range(len(fr.sources), world, rank)
    img, st = oracle.render_frame(fr, first_ray=first * fr.rays_per_source, ray_count=count * fr.rays_per_source,
                                  threads=1)
    t = torch.from_numpy(img.copy())
    allreduce_image(t)
    stats = torch.from_numpy(st.copy())
    dist.all_reduce(stats)
    if rank == 0:
        np.save(out_path, np.concatenate([t.numpy().ravel(), stats.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_single_render(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    out = str(tmp_path / "sum.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    fr = scenes.c0(scale=0.05, rays_per_source=30)[0]
    img, st = oracle.render_frame(fr)
    n = img.size
    assert np.array_equal(got[:n].reshape(img.shape), img)
    assert np.array_equal(got[n:], st)


def _bos_rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fr = scenes.c0(scale=0.01, rays_per_source=20)[0]
    med, opt = oracle.Medium.from_scene(fr.medium), oracle.Optics.from_scene(fr.optics)
    first, count = source_range(len(fr.sources), world, rank)
    _, disp, cnt = oracle.bos_displacements(med, opt, fr.sources, fr.rays_per_source, fr.seed, 0, fr.integrator,
                                            fr.step, threads=1, dot_ids=np.arange(first, first + count))
    # ranks' dot counts differ by at most one: pad to the largest, then gather
    m = source_range(len(fr.sources), world, 0)[1]
    pad = np.full((m, 3), np.nan)
    pad[:count, :2] = disp
    pad[:count, 2] = cnt
    parts = [torch.zeros((m, 3), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(pad))
    if rank == 0:
        rows = [p.numpy()[:source_range(len(fr.sources), world, r)[1]] for r, p in enumerate(parts)]
        np.save(out_path, np.concatenate(rows))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_bos_dots(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    out = str(tmp_path / "bos.npy")
    mp.spawn(_bos_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    fr = scenes.c0(scale=0.01, rays_per_source=20)[0]
    med, opt = oracle.Medium.from_scene(fr.medium), oracle.Optics.from_scene(fr.optics)
    _, disp, cnt = oracle.bos_displacements(med, opt, fr.sources, fr.rays_per_source, fr.seed, 0, fr.integrator,
                                            fr.step)
    assert np.array_equal(got[:, :2], disp, equal_nan=True)
    assert np.array_equal(got[:, 2].astype(np.int32), cnt)
