"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle on
the same seeded inputs.  Exit states: sensor position <= 1e-5 px, directions
<= 1e-6 rad, exit line <= 1e-5 px equivalent; images: relative L2 <= 1e-4
with exact 2^32-per-ray totals on both sides."""
import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes
from gpu_helpers import (compare_images, compare_states, gpu_handles, gpu_render, gpu_states, oracle_states,
                         vol_scale)

pytestmark = pytest.mark.gpu


def _all_ids(fr, limit=None):
    n = fr.n_rays if limit is None else min(limit, fr.n_rays)
    return np.arange(n, dtype=np.int64)


def _sample_ids(fr, n, seed=0):
    rng = np.random.default_rng(seed)
    return np.unique(rng.integers(0, fr.n_rays, n, dtype=np.int64))


@pytest.mark.parametrize("integ", [scenes.EULER, scenes.RK4])
def test_c0_states_and_image(integ):
    fr = scenes.c0(scale=0.1, rays_per_source=37)[0]   # 20x20 dots, ragged ray count
    fr.integrator = integ
    ids = _all_ids(fr)
    compare_states(gpu_states(fr, ids), oracle_states(fr, ids), fr.optics.pitch, vol_scale(fr))
    img_g, st_g = gpu_render(fr)
    img_o, st_o = oracle.render_frame(fr)
    compare_images(img_g, img_o, st_g, st_o, fr)


def test_c1_thick_lens_defocus():
    for fr in scenes.c1(scale=0.004):      # 40 particles, 400 rays, two frames
        ids = _all_ids(fr)
        compare_states(gpu_states(fr, ids), oracle_states(fr, ids), fr.optics.pitch, vol_scale(fr))
        img_g, st_g = gpu_render(fr)
        img_o, st_o = oracle.render_frame(fr)
        compare_images(img_g, img_o, st_g, st_o, fr)


def test_c2_turbulence_rk4_small_grid():
    fr = scenes.c2(scale=0.002, grid=64)[0]   # 200 dots x 200 rays
    ids = _all_ids(fr)
    res = compare_states(gpu_states(fr, ids), oracle_states(fr, ids), fr.optics.pitch, vol_scale(fr))
    assert res["n"] == fr.n_rays
    img_g, st_g = gpu_render(fr)
    img_o, st_o = oracle.render_frame(fr)
    compare_images(img_g, img_o, st_g, st_o, fr)


def test_c4_particles_inside_turbulence():
    fr = scenes.c4(scale=0.001, grid=48)[0]   # 100 particles x 1000 rays
    ids = _all_ids(fr)
    compare_states(gpu_states(fr, ids), oracle_states(fr, ids), fr.optics.pitch, vol_scale(fr))
    img_g, st_g = gpu_render(fr)
    img_o, st_o = oracle.render_frame(fr)
    compare_images(img_g, img_o, st_g, st_o, fr)


def test_c3_shock_gradient_turbulence_frames():
    frames = scenes.c3(scale=0.002, n_frames=3, max_grid=96)
    for fr in frames:
        ids = _all_ids(fr, limit=20000)
        compare_states(gpu_states(fr, ids), oracle_states(fr, ids), fr.optics.pitch, vol_scale(fr))


def test_full_size_c1_sampled_and_totals():
    """The benchmark workload at full size: sampled rays against the oracle,
    and the exact intensity total of the whole render."""
    frames = scenes.c1()
    for fr in frames:
        ids = _sample_ids(fr, 3000, seed=fr.frame_index)
        compare_states(gpu_states(fr, ids), oracle_states(fr, ids), fr.optics.pitch, vol_scale(fr))
        img_g, st_g = gpu_render(fr)
        assert st_g.sum() == fr.n_rays
        assert img_g.sum() == int(st_g[0]) << 32
        assert st_g[0] > 0.9 * fr.n_rays


def test_full_size_c2_sampled():
    fr = scenes.c2()[0]
    ids = _sample_ids(fr, 1500, seed=3)
    compare_states(gpu_states(fr, ids), oracle_states(fr, ids), fr.optics.pitch, vol_scale(fr))


def test_full_size_c4_sampled_and_totals():
    """The surrogate workload's plain render at full size (256^3 turbulence,
    1e9 rays, 2048^2 sensor): sampled rays against the oracle, and the exact
    intensity total of the whole render."""
    fr = scenes.c4()[0]
    ids = _sample_ids(fr, 1500, seed=5)
    compare_states(gpu_states(fr, ids), oracle_states(fr, ids), fr.optics.pitch, vol_scale(fr))
    img_g, st_g = gpu_render(fr)
    assert st_g.sum() == fr.n_rays
    assert img_g.sum() == int(st_g[0]) << 32
    assert st_g[0] > 0.5 * fr.n_rays
