"""Batched rendering (one persistent launch over frames of uneven size,
CUDA-graph replay) against the oracle's render of every frame and against
per-frame pivbos_render, and the autotuner."""
import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes
from gpu_helpers import compare_images, gpu_handles

pytestmark = pytest.mark.gpu


def _setup(frames):
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    hs = [gpu_handles(f) for f in frames]
    src = [torch.tensor(f.sources, dtype=torch.float64, device="cuda") for f in frames]
    imgs = [torch.zeros((f.optics.height, f.optics.width), dtype=torch.int64, device="cuda") for f in frames]
    stats = [torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device="cuda") for f in frames]
    descs = [P.frame_desc(h[0].h if h[0] else None, h[1].h, s, len(f.sources), f.rays_per_source, f.frame_index,
                          f.seed, f.step, im, st) for f, h, s, im, st in zip(frames, hs, src, imgs, stats)]
    return hs, src, imgs, stats, descs


def test_batch_matches_single_renders_and_graph_replay():
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    frames = scenes.c3(scale=0.002, n_frames=7, max_grid=96)
    hs, src, imgs, stats, descs = _setup(frames)
    ref, ref_st = [], []
    for f, h, s in zip(frames, hs, src):
        im = torch.zeros((f.optics.height, f.optics.width), dtype=torch.int64, device="cuda")
        st = torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device="cuda")
        P.pivbos_render(h[0].h, h[1].h, s, len(f.sources), f.rays_per_source, f.seed, f.frame_index,
                        f.integrator, f.step, im, st)
        ref.append(im)
        ref_st.append(st)
    for tuning in (None, P.pivbos_tuning(1024, 1, 2, 1), P.pivbos_tuning(512, 0, 3, 0)):
        for im, st in zip(imgs, stats):
            im.zero_()
            st.zero_()
        b = P.pivbos_batch_create(descs, scenes.RK4, tuning)
        try:
            P.pivbos_batch_render(b)
            P.pivbos_sync()
            for im, r, st, rs in zip(imgs, ref, stats, ref_st):
                assert torch.equal(im, r)
                assert torch.equal(st, rs)
            P.pivbos_batch_render(b)      # replay (graph when enabled)
            P.pivbos_sync()
            for im, r in zip(imgs, ref):
                assert torch.equal(im, 2 * r)
        finally:
            P.pivbos_batch_destroy(b)


@pytest.mark.parametrize("tuning", [None, (1024, 1, 2, 1), (512, 0, 3, 0)])
def test_batch_images_against_the_oracle(tuning):
    """Frames of uneven size (shock, gradient and turbulence fields, grids
    from 64^3) in one persistent launch: every frame's image and status
    counts against the oracle's render of that frame."""
    from paper_1812_05902_gb300 import pivbos as P
    frames = scenes.c3(scale=0.002, n_frames=5, max_grid=96)
    hs, src, imgs, stats, descs = _setup(frames)
    b = P.pivbos_batch_create(descs, scenes.RK4, P.pivbos_tuning(*tuning) if tuning else None)
    try:
        P.pivbos_batch_render(b)
        P.pivbos_sync()
    finally:
        P.pivbos_batch_destroy(b)
    for i, f in enumerate(frames):
        img_o, st_o = oracle.render_frame(f)
        st_g = stats[i].cpu().numpy()
        compare_images(imgs[i].cpu().numpy(), img_o, st_g, st_o, f, label="batch frame %d" % i)
        assert np.abs(st_g - st_o).sum() <= 2, (st_g, st_o)


def test_batch_rejects_host_buffers_and_bad_tuning():
    import ctypes
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    frames = scenes.c3(scale=0.001, n_frames=1, max_grid=64)
    hs, src, imgs, stats, descs = _setup(frames)
    host_img = np.zeros((1024, 1024), dtype=np.int64)
    bad = P.pivbos_frame_desc(*[getattr(descs[0], n) for n, _ in P.pivbos_frame_desc._fields_])
    bad.image = ctypes.c_void_p(host_img.ctypes.data)
    with pytest.raises(P.PivbosError):
        P.pivbos_batch_create([bad], scenes.RK4)
    with pytest.raises(P.PivbosError):
        P.pivbos_batch_create(descs, scenes.RK4, P.pivbos_tuning(300, 0, 3, 1))


def test_autotune_step_meets_tolerance():
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    from gpu_helpers import gpu_states
    fr = scenes.c2(scale=0.002, grid=64)[0]
    hs, src, imgs, stats, descs = _setup([fr])
    tol = 1e-3
    step, t = P.pivbos_autotune(descs[0], scenes.RK4, tol, 2048)
    assert fr.step / 64 <= step <= fr.step * 64
    assert t.rays_per_cta in (512, 1024, 2048) and t.cell_cache in (0, 1)
    # the chosen step's error, estimated the same way on other rays, is small
    ids = np.arange(0, fr.n_rays, max(1, fr.n_rays // 3000))[:3000]
    fr.step = step
    a = gpu_states(fr, ids, handles=hs[0])
    fr.step = step / 2
    b = gpu_states(fr, ids, handles=hs[0])
    ok = (a["status"] == 0) & (b["status"] == 0)
    err = np.max(np.abs(a["sensor_xy"][ok] - b["sensor_xy"][ok])) * 16 / 15
    assert err <= 4 * tol
