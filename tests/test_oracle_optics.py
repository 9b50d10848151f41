"""Pins for the oracle's optics (Sec. 3.3) and sensor (Sec. 3.4): the Snell
invariant of Eq. 7, sphere intersections against brute-force root finding,
ideal thin-lens conjugates, thick-lens paraxial imaging against an
independent ABCD computation, aperture and TIR kills."""
import math

import numpy as np
import pytest
import mpmath as mp

import oracle
from paper_1812_05902_gb300 import scenes


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def test_snell_tangential_invariant_and_unit_length():
    rng = np.random.default_rng(0)
    n_checked = 0
    for _ in range(2000):
        N = _unit(rng.normal(size=3))
        d = _unit(rng.normal(size=3))
        if N @ d > 0:
            N = -N
        n_i, n_f = rng.uniform(1.0, 1.8, 2)
        out = oracle.refract(d, N, n_i, n_f)
        sin_i = np.linalg.norm(np.cross(d, N))
        if n_i * sin_i > n_f:
            assert out is None       # total internal reflection
            continue
        n_checked += 1
        # Eq. 7: n_i sin(theta_i) = n_f sin(theta_f), as the full vector
        # identity n_i (d x N) = n_f (d' x N), and the ray stays in the plane
        np.testing.assert_allclose(n_i * np.cross(d, N), n_f * np.cross(out, N), atol=2e-15)
        assert abs(np.linalg.norm(out) - 1.0) < 1e-14
        assert out @ N < 0           # transmitted, not reflected
    assert n_checked > 1000


def test_refract_normal_incidence_and_identity():
    d = np.array([0.0, 0.0, 1.0])
    N = np.array([0.0, 0.0, -1.0])
    np.testing.assert_allclose(oracle.refract(d, N, 1.0, 1.5), d, atol=0)
    d2 = _unit([0.3, -0.2, 1.0])
    np.testing.assert_allclose(oracle.refract(d2, N, 1.3, 1.3), d2, atol=1e-16)


@pytest.mark.parametrize("R", [0.1, -0.1, 0.02, -0.5, 3.0])
def test_sphere_hit_against_brute_force(R):
    rng = np.random.default_rng(abs(int(R * 1000)))
    zv = 0.7
    C = np.array([0.0, 0.0, zv + R])
    for _ in range(200):
        P0 = np.array([rng.uniform(-0.003, 0.003), rng.uniform(-0.003, 0.003), zv - rng.uniform(0.05, 0.6)])
        d = _unit([rng.uniform(-0.005, 0.005), rng.uniform(-0.005, 0.005), 1.0])
        res = oracle.sphere_hit(P0, d, zv, R)
        assert res is not None
        P, N = res
        # brute force: bisection in 40-digit arithmetic on the distance to the
        # centre, bracketed between the vertex plane and 1.2 sags beyond it
        # (hit radius <= 6.5 mm by construction)
        mp.mp.dps = 40
        P0m = [mp.mpf(float(v)) for v in P0]
        dm = [mp.mpf(float(v)) for v in d]
        Cm = [mp.mpf(float(v)) for v in C]
        f = lambda t: mp.sqrt(sum((P0m[q] + t * dm[q] - Cm[q]) ** 2 for q in range(3))) - abs(mp.mpf(R))
        t_plane = (zv - P0[2]) / d[2]
        sag = 1.2 * (abs(R) - math.sqrt(R * R - 0.0065**2)) / d[2]
        lo, hi = (t_plane, t_plane + sag) if R > 0 else (t_plane - sag, t_plane)
        t = mp.findroot(f, (mp.mpf(lo), mp.mpf(hi)), solver="illinois")
        exp = np.array([float(P0m[q] + t * dm[q]) for q in range(3)])
        np.testing.assert_allclose(P, exp, rtol=0, atol=4e-16)
        # on the sphere, on the vertex-side cap, normal facing the ray
        assert abs(np.linalg.norm(P - C) - abs(R)) < 1e-15 * (1 + abs(R)) * 4
        assert (P[2] - C[2]) * R < 0
        assert abs(np.linalg.norm(N) - 1) < 1e-14 and N @ d < 0


def test_sphere_miss_outside_radius():
    # a ray parallel to the axis at radius larger than |R| cannot hit
    assert oracle.sphere_hit([0.2, 0.0, 0.0], [0.0, 0.0, 1.0], 0.5, 0.1) is None


def _optics(surfaces, n_object, aim_z, aim_r, sensor_z, W=512, H=512, pitch=10e-6, sigma=5e-6):
    rows = [s.as_row() for s in surfaces]
    return oracle.Optics(rows, n_object, aim_z, aim_r, sensor_z, pitch, W, H, sigma)


def test_ideal_thin_lens_conjugates_exact():
    f, M = 0.105, 0.1
    opt_s = scenes.ideal_lens_layout(0.0, M, f, 8.0, 1.00027, pitch=17e-6, width=256, height=256)
    opt = oracle.Optics.from_scene(opt_s)
    s_o = f * (1 + 1 / M)
    s_i = f * (1 + M)
    for src in ([0.0, 0.0, 0.0], [0.012, -0.007, 0.0], [-0.02, 0.02, 0.0]):
        xs = []
        for k in range(64):
            st = oracle.trace(None, opt, src, 9, 3, k, 0, oracle.EULER, 1e-4)
            assert st["status"] == oracle.REACHED
            xs.append(st["sensor_xy"])
        xs = np.array(xs)
        # every ray of a point source meets at one point, magnified by -s_i/s_o
        exp = np.array([-src[0] * s_i / s_o, -src[1] * s_i / s_o]) / 17e-6 + 128.0
        assert np.max(np.abs(xs - exp)) < 1e-7


def _abcd_image(R1, R2, d, ng, n0, s_o, h):
    """independent paraxial chief-ray calculation: image height and image
    distance after the rear vertex, by tracing two paraxial rays"""
    def trace(y, u):
        # (y, u) at the object plane, propagate s_o in n0
        y = y + u * s_o
        # surface 1
        u = (n0 * u - y * (ng - n0) / R1) / ng
        y = y + u * d
        u = (ng * u - y * (n0 - ng) / R2) / n0
        return y, u
    # marginal ray from the axis point sets the image distance
    y1, u1 = trace(0.0, 1e-4)
    s_i = -y1 / u1
    y2, u2 = trace(h, 0.0)
    return s_i, y2 + u2 * s_i


def test_thick_lens_paraxial_imaging():
    n0, ng = 1.000277, 1.5
    opt_s = scenes.thick_lens_layout(0.0, 0.2, 4.0, n0, width=1024, height=1024)
    zv1 = opt_s.surfaces[1].z
    s_o = zv1 - 0.0
    s_i_exp, _ = _abcd_image(0.1, -0.1, 0.01, ng, n0, s_o, 0.0)
    assert abs((opt_s.sensor_z - opt_s.surfaces[2].z) - s_i_exp) < 1e-9
    # shrink the aperture so that only paraxial rays pass
    opt_s.aim_r = 0.05e-3
    opt_s.surfaces[0].clear_r = 0.05e-3
    opt = oracle.Optics.from_scene(opt_s)
    for h in (0.0, 2e-3, -5e-3):
        _, y_img = _abcd_image(0.1, -0.1, 0.01, ng, n0, s_o, h)
        pts = []
        for k in range(32):
            st = oracle.trace(None, opt, [0.0, h, 0.0], 1, 0, k, 0, oracle.EULER, 1e-4)
            assert st["status"] == oracle.REACHED
            pts.append(st["sensor_xy"][1])
        y = (np.mean(pts) - 512.0) * 17e-6
        assert abs(y - y_img) < 2e-3 * 17e-6 + 1e-4 * abs(h) ** 3 / 0.1**2
        assert abs(y_img / h + 0.2) < 1e-6 if h else True


def test_aperture_blocks_rays_outside_the_stop():
    n0 = 1.0
    surfaces = [scenes.Surface(scenes.STOP, 1.0, clear_r=0.005),
                scenes.Surface(scenes.IDEAL_THIN, 1.0, f=0.1, n_after=n0, clear_r=0.1)]
    # aim at a disk twice as large as the stop: a quarter of the rays pass
    opt = _optics(surfaces, n0, 1.0, 0.01, 1.111111111)
    n = 4000
    st = oracle.trace_many(None, opt, np.array([[0.0, 0.0, 0.0]]), n, np.arange(n), 4, 0, oracle.EULER, 1e-4)
    passed = np.mean(st["status"] == oracle.REACHED)
    assert set(np.unique(st["status"])) <= {oracle.REACHED, oracle.KILLED_STOP}
    assert abs(passed - 0.25) < 4 * math.sqrt(0.25 * 0.75 / n)


def test_total_internal_reflection_kills():
    # a flat glass->air exit face hit at 60 degrees from glass (n = 1.5):
    # sin(60) * 1.5 > 1 so the ray must be killed by TIR
    n0 = 1.0
    surfaces = [scenes.Surface(scenes.PLANE, 1.0, n_after=1.5, clear_r=10.0),
                scenes.Surface(scenes.PLANE, 1.5, n_after=1.0, clear_r=10.0)]
    opt = _optics(surfaces, 1.5, 1.0, 1e-9, 2.0)
    src = [-math.tan(math.radians(60.0)) * 1.0, 0.0, 0.0]
    st = oracle.trace(None, opt, src, 0, 0, 0, 0, oracle.EULER, 1e-4)
    assert st["status"] == oracle.KILLED_TIR
    src2 = [-math.tan(math.radians(30.0)) * 1.0, 0.0, 0.0]
    st2 = oracle.trace(None, opt, src2, 0, 0, 0, 0, oracle.EULER, 1e-4)
    assert st2["status"] != oracle.KILLED_TIR


def test_off_sensor_rays_do_not_reach():
    f, M = 0.105, 0.1
    opt_s = scenes.ideal_lens_layout(0.0, M, f, 8.0, 1.0, pitch=17e-6, width=64, height=64)
    opt = oracle.Optics.from_scene(opt_s)
    # the image of this source lies beyond the 64-pixel array
    st = oracle.trace(None, opt, [0.02, 0.0, 0.0], 0, 0, 0, 0, oracle.EULER, 1e-4)
    assert st["status"] == oracle.KILLED_OFF_SENSOR
