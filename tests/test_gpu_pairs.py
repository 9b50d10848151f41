"""GPU parity of the image-pair helpers through the C ABI: particles moved by
a velocity field (pivbos_advect_sources) and the 16-bit image
(pivbos_image_u16), against the CPU FP64 oracle; and a rendered pair whose
particle images move as the optics predict."""
import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes
from gpu_helpers import gpu_render

pytestmark = pytest.mark.gpu


def test_advect_matches_oracle():
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    rng = np.random.default_rng(8)
    nz, ny, nx = 9, 12, 15
    vel = rng.normal(0.0, 2.0, (nz, ny, nx, 3)).astype(np.float32)
    origin, spacing = (-0.02, -0.03, 0.1), (0.003, 0.005, 0.004)
    lo = np.array(origin) - 0.005
    hi = np.array(origin) + np.array(spacing) * (np.array([nx, ny, nz]) - 1) + 0.005
    src = lo + (hi - lo) * rng.random((5001, 3))          # some outside the grid (clamped)
    dt = 1e-3
    exp = oracle.advect(src, vel, origin, spacing, dt)
    s = torch.tensor(src, device="cuda")
    out = torch.empty_like(s)
    P.pivbos_advect_sources(s, len(src), torch.tensor(vel, device="cuda"), origin, spacing, dt, out)
    P.pivbos_sync()
    np.testing.assert_allclose(out.cpu().numpy(), exp, rtol=0, atol=1e-15)


def test_u16_matches_oracle_bit_for_bit():
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    fr = scenes.c0(scale=0.05, rays_per_source=60)[0]
    img, _ = gpu_render(fr)
    for full_scale in (float(img.max()) / 2 ** 32 * 0.5, 60.0, 1e4):       # saturating, partial, faint
        for n in (img.size, 1001, 7):                                      # 8-pixel groups and ragged tails
            flat = np.ascontiguousarray(img.ravel()[:n])
            g = torch.empty(n, dtype=torch.int16, device="cuda")     # the kernel writes raw 16-bit words
            P.pivbos_image_u16(torch.tensor(flat, device="cuda"), n, full_scale, g)
            P.pivbos_sync()
            got = g.cpu().numpy().view(np.uint16)
            assert np.array_equal(got, oracle.image_u16(flat, full_scale))
    assert (oracle.image_u16(img, float(img.max()) / 2 ** 32 * 0.5) == 65535).any()


def test_rendered_pair_moves_with_the_flow():
    """A uniform flow moves every particle by D; in the C1 camera (M = 0.2,
    inverted real image, unflipped sensor frame) the intensity centroid of
    the second image sits -M D / pitch from the first's."""
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    fr = scenes.c1(scale=0.01)[0]                       # 100 particles x 1e4 rays (scale 0.01 -> 1e4)
    fr.rays_per_source = 400
    U = np.array([0.3, -0.2, 0.0])                      # m/s
    dt = 1e-3                                           # D = (0.3, -0.2) mm
    vel = np.ascontiguousarray(np.tile(U, (4, 4, 4, 1)), dtype=np.float32)
    src = torch.tensor(fr.sources, device="cuda")
    moved = torch.empty_like(src)
    P.pivbos_advect_sources(src, len(fr.sources), torch.tensor(vel, device="cuda"), (-0.03, -0.03, -0.01),
                            (0.02, 0.02, 0.01), dt, moved)
    P.pivbos_sync()
    fr_b = scenes.Frame(fr.medium, fr.optics, moved.cpu().numpy(), fr.rays_per_source, fr.seed, fr.integrator,
                        fr.step, fr.frame_index + 1)
    a, _ = gpu_render(fr)
    b, _ = gpu_render(fr_b)

    def centroid(im):
        w = im.astype(np.float64)
        y, x = np.indices(im.shape)
        return np.array([(w * x).sum(), (w * y).sum()]) / w.sum()

    shift = centroid(b) - centroid(a)
    exp = -fr.optics.magnification * U[:2] * dt / fr.optics.pitch
    np.testing.assert_allclose(shift, exp, rtol=0.03)
