"""One image sharded across ranks through the product library: two
processes (gloo; both on the one GPU this runs on -- their kernels never
wait on one another) each render a contiguous range of the sources with the
global source indices, through the plain path (pivbos_render_range) and the
surrogate path (pivbos_surrogate_render_range), and one all-reduce sums the
int64 fixed-point images.  The sums must equal the single-process renders
bit for bit: integer addition is exact in any order."""
import os
import socket

import numpy as np
import pytest

from paper_1812_05902_gb300 import scenes
from paper_1812_05902_gb300.shard import allreduce_image, source_range

pytestmark = pytest.mark.gpu


def _frame():
    return scenes.c4(scale=0.002, grid=64)[0]      # 200 particles x 2000 rays in a 64^3 field


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _setup(fr, sources, P, torch):
    from gpu_helpers import gpu_handles
    med, opt = gpu_handles(fr)
    src = torch.tensor(sources, dtype=torch.float64, device="cuda")
    img = torch.zeros((fr.optics.height, fr.optics.width), dtype=torch.int64, device="cuda")
    st = torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device="cuda")
    return med, opt, src, img, st


def _surrogate_cfg(P):
    cfg = P.pivbos_surrogate_default_cfg()
    cfg.use_network = 0            # the projection: the same surrogate on every rank
    cfg.n_val = 400_000
    cfg.min_bin_count = 1
    cfg.err_budget_px = 1.0        # every bin served: no budget decision near a tie
    return cfg


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    from paper_1812_05902_gb300 import pivbos as P
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fr = _frame()
    first, count = source_range(len(fr.sources), world, rank)
    med, opt, src_all, img, st = _setup(fr, fr.sources, P, torch)
    src = src_all[first:first + count].contiguous()
    P.pivbos_render_range(med.h, opt.h, src, count, first, fr.rays_per_source, fr.seed, fr.frame_index,
                          fr.integrator, fr.step, img, st)
    # the surrogate trained on the whole frame, rendered for this rank's range
    img_s = torch.zeros_like(img)
    st_s = torch.zeros_like(st)
    desc_all = P.frame_desc(med.h, opt.h, src_all, len(fr.sources), fr.rays_per_source, fr.frame_index, fr.seed,
                            fr.step, img_s, st_s)
    desc = P.frame_desc(med.h, opt.h, src, count, fr.rays_per_source, fr.frame_index, fr.seed, fr.step, img_s, st_s)
    sg, _ = P.pivbos_surrogate_train(desc_all, fr.integrator, _surrogate_cfg(P))
    try:
        P.pivbos_surrogate_render_range(sg, desc, first)
        P.pivbos_sync()
    finally:
        P.pivbos_surrogate_destroy(sg)
    parts = [img.cpu(), st.cpu(), img_s.cpu(), st_s.cpu()]
    for t in parts:
        allreduce_image(t)            # gloo: host tensors
    if rank == 0:
        np.savez(out_path, *[t.numpy() for t in parts])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sum_to_the_single_gpu_images(tmp_path):
    import torch
    import torch.multiprocessing as mp
    from paper_1812_05902_gb300 import pivbos as P
    out = str(tmp_path / "sum.npz")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    fr = _frame()
    med, opt, src, img, st = _setup(fr, fr.sources, P, torch)
    P.pivbos_render(med.h, opt.h, src, len(fr.sources), fr.rays_per_source, fr.seed, fr.frame_index,
                    fr.integrator, fr.step, img, st)
    img_s = torch.zeros_like(img)
    st_s = torch.zeros_like(st)
    desc = P.frame_desc(med.h, opt.h, src, len(fr.sources), fr.rays_per_source, fr.frame_index, fr.seed, fr.step,
                        img_s, st_s)
    sg, rep = P.pivbos_surrogate_train(desc, fr.integrator, _surrogate_cfg(P))
    try:
        P.pivbos_surrogate_render(sg, desc)
        P.pivbos_sync()
    finally:
        P.pivbos_surrogate_destroy(sg)
    assert rep.val_served_frac > 0.99
    assert int(st.cpu().sum()) == fr.n_rays
    assert np.array_equal(got["arr_0"], img.cpu().numpy())
    assert np.array_equal(got["arr_1"], st.cpu().numpy())
    assert np.array_equal(got["arr_2"], img_s.cpu().numpy())
    assert np.array_equal(got["arr_3"], st_s.cpu().numpy())
