"""The extended optics (mirrors, lens arrays, a turned sensor, Mie radiance)
on the other render paths: the persistent batch kernel against per-frame
renders (bit for bit), and the surrogate path (its finish kernel and the
fallback list) against the plain render."""
import dataclasses

import numpy as np
import pytest

from paper_1812_05902_gb300 import scenes
from gpu_helpers import gpu_handles

pytestmark = pytest.mark.gpu


def _variant(fr, kind):
    o = fr.optics
    if kind == "mie":
        fr.optics = dataclasses.replace(o, mie=scenes.Mie())
    elif kind == "plenoptic":
        fr.optics = dataclasses.replace(o, surfaces=list(o.surfaces) + [
            scenes.Surface(scenes.LENS_ARRAY, o.sensor_z - 5e-4, R=1e-4, f=5e-4, clear_r=0.05)])
    elif kind == "tilted":
        fr.optics = dataclasses.replace(o, sensor_tilt_x=0.05, sensor_tilt_y=-0.03)
    return fr


def test_batch_with_extended_optics_matches_single_renders():
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    frames = scenes.c3(scale=0.002, n_frames=4, max_grid=64)
    for fr, kind in zip(frames, ("mie", "plenoptic", "tilted", "plain")):
        _variant(fr, kind)
    hs = [gpu_handles(f) for f in frames]
    src = [torch.tensor(f.sources, dtype=torch.float64, device="cuda") for f in frames]
    imgs = [torch.zeros((f.optics.height, f.optics.width), dtype=torch.int64, device="cuda") for f in frames]
    descs = [P.frame_desc(h[0].h, h[1].h, s, len(f.sources), f.rays_per_source, f.frame_index, f.seed, f.step, im)
             for f, h, s, im in zip(frames, hs, src, imgs)]
    ref, ref_st = [], []
    for f, h, s in zip(frames, hs, src):
        im = torch.zeros((f.optics.height, f.optics.width), dtype=torch.int64, device="cuda")
        st = torch.zeros(P.RAY_NSTATUS, dtype=torch.int64, device="cuda")
        P.pivbos_render(h[0].h, h[1].h, s, len(f.sources), f.rays_per_source, f.seed, f.frame_index,
                        f.integrator, f.step, im, st)
        ref.append(im)
        ref_st.append(st)
    b = P.pivbos_batch_create(descs, scenes.RK4)
    try:
        P.pivbos_batch_render(b)
        P.pivbos_sync()
        for im, r in zip(imgs, ref):
            assert torch.equal(im, r)
        # the Mie frame's rays weigh less than 1, the others exactly 1
        assert ref[0].sum().item() < 0.9 * (int(ref_st[0][0].item()) << 32)
        for k in (1, 2, 3):
            assert ref[k].sum().item() == int(ref_st[k][0].item()) << 32
    finally:
        P.pivbos_batch_destroy(b)


@pytest.mark.parametrize("kind", ["mie", "tilted"])
def test_surrogate_with_extended_optics(kind):
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    frame = _variant(scenes.c4(scale=0.001, grid=64)[0], kind)
    med, opt = gpu_handles(frame)
    src = torch.tensor(frame.sources, dtype=torch.float64, device="cuda")
    img = torch.zeros((frame.optics.height, frame.optics.width), dtype=torch.int64, device="cuda")
    desc = P.frame_desc(med.h, opt.h, src, len(frame.sources), frame.rays_per_source, frame.frame_index,
                        frame.seed, frame.step, img)
    ref = torch.zeros_like(img)
    P.pivbos_render(med.h, opt.h, src, len(frame.sources), frame.rays_per_source, frame.seed, frame.frame_index,
                    frame.integrator, frame.step, ref)
    for budget in (1e-12, 0.01):          # everything to the fallback list, then a served map
        cfg = P.pivbos_surrogate_default_cfg()
        cfg.n_train = 1_000_000
        cfg.n_val = 500_000
        cfg.epochs = 4
        cfg.err_budget_px = budget
        sg, rep = P.pivbos_surrogate_train(desc, frame.integrator, cfg)
        try:
            img.zero_()
            n_fb = P.pivbos_surrogate_render(sg, desc, count_fallback=True)
            P.pivbos_sync()
            if budget < 1e-9:
                assert n_fb == frame.n_rays
                assert torch.equal(img, ref)
            else:
                assert n_fb < 0.5 * frame.n_rays
                a, b = img.double(), ref.double()
                assert (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item() < 0.05
                assert abs(a.sum().item() / b.sum().item() - 1.0) < 1e-3
        finally:
            P.pivbos_surrogate_destroy(sg)
