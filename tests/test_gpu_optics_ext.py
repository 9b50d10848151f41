"""GPU parity of the optical extensions of Sec. 3.3-3.4 through the C ABI:
a camera built around a concave mirror (law of reflection, the system
unfolded at the mirror) behind a flat fold mirror, a plenoptic camera (the
thick lens of C1 with an array of lenslets in front of the sensor), and a
sensor turned about its centre (Fig. 1(d), Scheimpflug), each with rays
through a density field.  Against the CPU FP64 oracle on the same seeded
inputs: sensor positions <= 1e-5 px, directions <= 1e-6 rad, images
relative L2 <= 1e-4 with exact 2^32-per-ray totals."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes
from gpu_helpers import compare_images, compare_states, gpu_render, gpu_states, oracle_states, vol_scale

pytestmark = pytest.mark.gpu


def _mirror_camera():
    fr = scenes.c0(scale=0.02, rays_per_source=53)[0]      # 9 x 9 dots, C0 slab, Euler
    n0 = fr.optics.n_object
    zs, zv, R = 1.15, 1.16, -0.2
    s_o = zv
    s_i = 1.0 / (2.0 / abs(R) - 1.0 / s_o)
    a = 6.5e-3
    surf = [scenes.Surface(scenes.MIRROR, 1.0, R=0.0, clear_r=0.05),          # flat fold mirror
            scenes.Surface(scenes.STOP, zs, clear_r=a),
            scenes.Surface(scenes.MIRROR, zv, R=R, clear_r=0.02)]
    fr.optics = scenes.Optics(surfaces=surf, n_object=n0, aim_z=zs, aim_r=a, sensor_z=zv + s_i, pitch=17e-6,
                              width=256, height=256, f_number=8.0, magnification=s_i / s_o)
    return fr


def _plenoptic():
    fr = scenes.c1(scale=0.003)[0]                          # 30 particles x 300 rays
    o = fr.optics
    surf = list(o.surfaces) + [scenes.Surface(scenes.LENS_ARRAY, o.sensor_z - 5e-4, R=1e-4, f=5e-4,
                                              clear_r=0.05)]
    fr.optics = dataclasses.replace(o, surfaces=surf)
    return fr


def _tilted():
    fr = scenes.c0(scale=0.02, rays_per_source=41)[0]
    fr.integrator = scenes.RK4
    fr.optics = dataclasses.replace(fr.optics, sensor_tilt_x=0.12, sensor_tilt_y=-0.07)
    return fr


@pytest.mark.parametrize("make", [_mirror_camera, _plenoptic, _tilted], ids=["mirror", "plenoptic", "tilted"])
def test_optics_extensions_match_oracle(make):
    fr = make()
    ids = np.arange(fr.n_rays, dtype=np.int64)
    g = gpu_states(fr, ids)
    o = oracle_states(fr, ids)
    res = compare_states(g, o, fr.optics.pitch, vol_scale(fr))
    assert res["reached"] > 0.5 * fr.n_rays, res
    img_g, st_g = gpu_render(fr)
    img_o, st_o = oracle.render_frame(fr)
    compare_images(img_g, img_o, st_g, st_o, fr)


def test_mirror_camera_focuses_and_plenoptic_splits():
    """Behaviour the extensions exist for: the mirror camera images a dot to
    a point (rays of one dot within a pixel through the uniform medium), and
    the lenslets cut one particle's light into many separate spots."""
    fr = _mirror_camera()
    fr.medium = None
    ids = np.arange(fr.rays_per_source, dtype=np.int64)
    st = gpu_states(fr, ids)
    ok = st["status"] == oracle.REACHED
    assert ok.sum() > 0.9 * len(ids)
    assert np.ptp(st["sensor_xy"][ok], axis=0).max() < 1.0      # a corner dot: off-axis aberrations only
    fr = _plenoptic()
    ids = np.arange(fr.rays_per_source, dtype=np.int64)
    st = gpu_states(fr, ids)
    ok = st["status"] == oracle.REACHED
    cells = {tuple(np.floor(p / 5.88).astype(int)) for p in st["sensor_xy"][ok]}    # 100 um lenslets = 5.88 px
    assert len(cells) > 10
