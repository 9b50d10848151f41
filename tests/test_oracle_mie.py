"""Pins for the oracle's Mie radiance (Sec. 3.1: rays of a PIV particle carry
the radiance Mie scattering gives, computed with the method of Bohren &
Huffman): the Rayleigh limit's closed forms, energy conservation for a
non-absorbing sphere, the optical theorem, the angular normalisation of the
scattered intensity, the large-sphere extinction limit, the dipole pattern
of a polarised laser, and the exact intensity total of a weighted render."""
import math

import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes


@pytest.mark.parametrize("m", [1.33, 1.5, 2.0])
def test_rayleigh_limit(m):
    x = 0.01
    s12, q = oracle.mie(x, m, 0.0, 181)
    K = (m * m - 1.0) / (m * m + 2.0)
    np.testing.assert_allclose(q["q_sca"], 8.0 / 3.0 * x ** 4 * K * K, rtol=1e-3)
    th = np.linspace(0.0, np.pi, 181)
    # |S1|^2 = x^6 K^2 at every angle, |S2|^2 = |S1|^2 cos^2(theta)
    np.testing.assert_allclose(s12[:, 0], x ** 6 * K * K, rtol=1e-3)
    np.testing.assert_allclose(s12[:, 1], s12[:, 0] * np.cos(th) ** 2, rtol=0, atol=1e-3 * x ** 6 * K * K)


@pytest.mark.parametrize("x", [0.5, 5.905, 50.0, 300.0])
@pytest.mark.parametrize("m", [1.33, 1.5, 2.0])
def test_energy_conservation_and_optical_theorem(x, m):
    s12, q = oracle.mie(x, m, 0.0, 3)
    # a non-absorbing sphere scatters all it removes
    np.testing.assert_allclose(q["q_ext"], q["q_sca"], rtol=1e-10)
    # optical theorem: Q_ext = (4 / x^2) Re S(0)
    np.testing.assert_allclose(q["q_ext"], 4.0 / (x * x) * q["re_s0"], rtol=1e-10)
    assert q["terms"] == int(x + 4.0 * x ** (1.0 / 3.0) + 2.0)
    # forward and backward: S1 = +-S2
    np.testing.assert_allclose(s12[0, 0], s12[0, 1], rtol=1e-12)
    np.testing.assert_allclose(s12[-1, 0], s12[-1, 1], rtol=1e-8)


@pytest.mark.parametrize("x,m", [(1.0, 1.5), (5.905, 1.45), (20.0, 1.33), (8.0, 1.5 + 0.05j)])
def test_scattered_intensity_integrates_to_q_sca(x, m):
    n = 40001
    s12, q = oracle.mie(x, m.real, m.imag, n)
    th = np.linspace(0.0, np.pi, n)
    f = (s12[:, 0] + s12[:, 1]) * np.sin(th)
    h = th[1] - th[0]
    simpson = h / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum())
    np.testing.assert_allclose(simpson / (x * x), q["q_sca"], rtol=1e-7)


def test_absorbing_spheres():
    _, q = oracle.mie(8.0, 1.5, 0.1, 3)
    assert q["q_ext"] > q["q_sca"] > 0.0
    np.testing.assert_allclose(q["q_ext"], 4.0 / 64.0 * q["re_s0"], rtol=1e-10)
    # extinction paradox: a large sphere removes twice its geometric cross-section
    _, q = oracle.mie(1000.0, 1.5, 0.5, 3)
    assert abs(q["q_ext"] - 2.0) < 0.02


def _opt_with_radiance(x, m, pol):
    o = oracle.Optics(np.zeros((0, 6)), 1.0, 1.0, 1e-3, 1.1, 1e-5, 1024, 1024, 1e-5)
    s12, _ = oracle.mie(x, m, 0.0, 721)
    return o.radiance(s12, (1.0, 0.0, 0.0), pol), s12


def test_polarised_dipole_pattern():
    """A small particle lit by a laser along x polarised along z radiates
    nothing along z and the most along y; unpolarised light halves the
    intensity at 90 degrees."""
    o, s12 = _opt_with_radiance(0.01, 1.5, (0.0, 0.0, 1.0))
    # a source at the origin, lens disk tiny around (0, 0, 1): rays along +z
    w = oracle.ray_weight(o, [0.0, 0.0, 0.0], 0, 0, 0, 0)
    assert w < 1e-6
    o, _ = _opt_with_radiance(0.01, 1.5, (0.0, 1.0, 0.0))
    w = oracle.ray_weight(o, [0.0, 0.0, 0.0], 0, 0, 0, 0)
    np.testing.assert_allclose(w, 1.0, rtol=1e-4)
    o, _ = _opt_with_radiance(0.01, 1.5, None)
    w = oracle.ray_weight(o, [0.0, 0.0, 0.0], 0, 0, 0, 0)
    np.testing.assert_allclose(w, 0.5, rtol=1e-3)


def test_weighted_render_total_is_exact():
    fr = scenes.c1(scale=0.001)[0]          # 10 particles x 100 rays
    fr.optics.mie = scenes.Mie()
    med = oracle.Medium.from_scene(fr.medium)
    opt = oracle.Optics.from_scene(fr.optics)
    img, st = oracle.render(med, opt, fr.sources, fr.rays_per_source, fr.seed, fr.frame_index, fr.integrator,
                            fr.step)
    ids = np.arange(fr.n_rays)
    states = oracle.trace_many(med, opt, fr.sources, fr.rays_per_source, ids, fr.seed, fr.frame_index,
                               fr.integrator, fr.step)
    total = 0
    ws = []
    for r in ids[states["status"] == oracle.REACHED]:
        s, k = divmod(int(r), fr.rays_per_source)
        w = oracle.ray_weight(opt, fr.sources[s], fr.seed, s, k, fr.frame_index)
        ws.append(w)
        total += int(np.rint(w * 2.0 ** 32))
    assert img.sum() == total
    assert 0.0 < min(ws) and max(ws) <= 1.0
    assert max(ws) / min(ws) > 1.01         # the radiance varies across the lens
