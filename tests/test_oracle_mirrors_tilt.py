"""Pins for the oracle's optical extensions of Sec. 3.3-3.4: mirrors (the law
of reflection, item 1), arrays of lenses (the plenoptic camera of item 2)
and a sensor that is not square to the axis (Fig. 1(d), perspective and the
Scheimpflug arrangement).  Each is checked against geometry written out in
the test: the reflection invariants, the exact axis crossing of a ray
reflected by a sphere, the mirror and thin-lens equations, and the
Scheimpflug condition of an ideal lens."""
import math

import numpy as np

import oracle

W = H = 2048
PITCH = 1e-6


def _optics(rows, sensor_z, aim_z=0.0, aim_r=1e-3, n_object=1.0, w=W, h=H, pitch=PITCH):
    return oracle.Optics(np.array(rows, dtype=np.float64).reshape(-1, 6), n_object, aim_z, aim_r, sensor_z,
                         pitch, w, h, 1e-6)


def test_law_of_reflection_invariants():
    rng = np.random.default_rng(1)
    for _ in range(200):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        N = rng.normal(size=3)
        N /= np.linalg.norm(N)
        r = oracle.reflect(d, N)
        assert abs(np.linalg.norm(r) - 1.0) < 2e-15
        assert abs(r @ N + d @ N) < 2e-15                   # angle in = angle out
        assert np.linalg.norm(np.cross(r - d, N)) < 4e-15    # change along the normal only
        assert abs(np.cross(d, N) @ r) < 4e-15               # in the plane of incidence


def test_flat_mirror_unfolds_to_nothing():
    P = np.array([1e-4, -2e-4, 0.0])
    d = np.array([1e-4, 2e-4, 1.0])
    d /= np.linalg.norm(d)
    plain = oracle.trace_optics(_optics(np.zeros((0, 6)), 1.0), P, d)
    mirror = oracle.trace_optics(_optics([[oracle.MIRROR, 0.4, 0.0, 0.0, 1.0, 0.1]], 1.0), P, d)
    assert plain["status"] == mirror["status"] == oracle.REACHED
    np.testing.assert_array_equal(plain["sensor_xy"], mirror["sensor_xy"])
    # outside the clear radius: a miss
    small = oracle.trace_optics(_optics([[oracle.MIRROR, 0.4, 0.0, 0.0, 1.0, 1e-5]], 1.0), P, d)
    assert small["status"] == oracle.KILLED_MISS


def test_concave_mirror_axis_crossing_exact():
    """A ray parallel to the axis at height h, reflected by a sphere of
    radius |R|, crosses the axis |R| / (2 cos theta) from the centre,
    sin theta = h / |R|; unfolded, that is z_v + |R| - |R| / (2 cos theta)."""
    zv, R = 1.0, -0.4                      # centre at zv + R, on the incoming side: concave
    for h in (1e-4, 5e-3, 0.02, 0.08, 0.15):
        th = math.asin(h / abs(R))
        zc = zv + abs(R) - abs(R) / (2.0 * math.cos(th))
        opt = _optics([[oracle.MIRROR, zv, R, 0.0, 1.0, 0.3]], zc)
        st = oracle.trace_optics(opt, [0.0, h, 0.0], [0.0, 0.0, 1.0])
        assert st["status"] == oracle.REACHED
        assert abs(st["sensor_xy"][1] - H / 2) < 1e-6, (h, st["sensor_xy"])
        assert st["sensor_xy"][0] == W / 2
        # after the mirror the unfolded ray heads down to the axis
        assert st["sensor_dir"][2] > 0 and st["sensor_dir"][1] < 0


def test_mirror_equation_paraxial_point_source():
    """1/s_o + 1/s_i = 2/|R| and magnification -s_i/s_o for a concave
    mirror, rays within a tiny stop."""
    zv, R = 0.5, -0.3
    s_o = 0.5
    s_i = 1.0 / (2.0 / abs(R) - 1.0 / s_o)
    h = 2e-4
    # the stop sits before the mirror's sag (a concave mirror bends back
    # toward the incoming light off the axis)
    rows = [[oracle.STOP, zv - 0.01, 0.0, 0.0, 1.0, 5e-5], [oracle.MIRROR, zv, R, 0.0, 1.0, 0.1]]
    opt = _optics(rows, zv + s_i, aim_z=zv - 0.01, aim_r=5e-5)
    hits = np.array([oracle.trace(None, opt, [0.0, h, 0.0], 3, 0, k, 0, oracle.RK4, 1e-3)["sensor_xy"]
                     for k in range(64)])
    y = (hits[:, 1] - H / 2) * PITCH
    np.testing.assert_allclose(y, -h * s_i / s_o, rtol=2e-6)


def test_lens_array_images_through_each_lenslet():
    """Every ray of a point source meets, behind lenslet c, at the image
    c - (s_i / s_o)(h - c) of the thin-lens equation."""
    za, f, p = 0.2, 0.01, 2e-3
    s_o = 0.2
    s_i = 1.0 / (1.0 / f - 1.0 / s_o)
    src = np.array([3e-4, -7e-4, 0.0])
    rows = [[oracle.LENS_ARRAY, za, p, f, 1.0, 0.05]]
    opt = _optics(rows, za + s_i, aim_z=za, aim_r=6e-3, pitch=1e-6, w=20000, h=20000)
    seen = set()
    for k in range(400):
        st = oracle.trace(None, opt, src, 11, 0, k, 0, oracle.RK4, 1e-3)
        lp = oracle.lens_point(11, 0, k, 0, 6e-3, za)
        c = p * np.floor(lp[:2] / p + 0.5)
        seen.add(tuple(np.round(c / p).astype(int)))
        img = c - (s_i / s_o) * (src[:2] - c)
        assert st["status"] == oracle.REACHED
        np.testing.assert_allclose((st["sensor_xy"] - 10000.0) * 1e-6, img, rtol=0, atol=1e-12)
    assert len(seen) >= 20                 # many lenslets were used


def _ideal_lens(zl, f, a):
    return [[oracle.STOP, zl, 0.0, 0.0, 1.0, a], [oracle.IDEAL_THIN, zl, 0.0, f, 1.0, 1.5 * a]]


def test_tilted_sensor_zero_tilt_is_the_plain_sensor():
    rows = _ideal_lens(1.0, 0.1, 5e-3)
    a = _optics(rows, 1.12, aim_z=1.0, aim_r=5e-3)
    b = _optics(rows, 1.12, aim_z=1.0, aim_r=5e-3).tilt_sensor(0.0, 0.0)
    for k in range(16):
        sa = oracle.trace(None, a, [1e-3, 2e-3, 0.0], 1, 0, k, 0, oracle.RK4, 1e-3)
        sb = oracle.trace(None, b, [1e-3, 2e-3, 0.0], 1, 0, k, 0, oracle.RK4, 1e-3)
        np.testing.assert_array_equal(sa["sensor_xy"], sb["sensor_xy"])


def test_scheimpflug_tilted_object_plane_is_sharp_on_the_tilted_sensor():
    """An ideal thin lens maps planes to planes: an object plane tilted by
    alpha about x images onto a plane through the axial image point; a
    sensor turned to it (tan t = dz'/dy' of two image points) receives every
    ray of every source on the object plane at one point, the image the
    thin-lens equation gives."""
    zl, f, a = 1.0, 0.1, 5e-3
    z0 = 0.0
    alpha = 0.4

    def image(x, y):
        s = zl - (z0 + y * math.tan(alpha))
        si = s * f / (s - f)
        return np.array([-x * si / s, -y * si / s, zl + si])

    i0, i1 = image(0.0, 0.0), image(0.0, 0.01)
    t = math.atan((i1[2] - i0[2]) / (i1[1] - i0[1]))
    pitch = 1e-6
    opt = _optics(_ideal_lens(zl, f, a), i0[2], aim_z=zl, aim_r=a, w=8000, h=8000, pitch=pitch)
    opt.tilt_sensor(t, 0.0)
    ev = np.array([0.0, math.cos(t), math.sin(t)])
    spreads = []
    for (x, y) in ((0.0, 0.0), (0.004, 0.006), (-0.007, -0.009), (0.01, 0.012)):
        src = [x, y, z0 + y * math.tan(alpha)]
        hits = np.array([oracle.trace(None, opt, src, 2, 0, k, 0, oracle.RK4, 1e-3)["sensor_xy"] for k in range(48)])
        im = image(x, y)
        exp = np.array([im[0] / pitch + 4000.0, (im - i0) @ ev / pitch + 4000.0])
        np.testing.assert_allclose(hits, np.broadcast_to(exp, hits.shape), rtol=0, atol=1e-6)
        spreads.append(np.ptp(hits, axis=0).max())
    # the same sources on a sensor square to the axis are blurred off-axis
    flat = _optics(_ideal_lens(zl, f, a), i0[2], aim_z=zl, aim_r=a, w=8000, h=8000, pitch=pitch)
    src = [0.0, 0.012, z0 + 0.012 * math.tan(alpha)]
    hits = np.array([oracle.trace(None, flat, src, 2, 0, k, 0, oracle.RK4, 1e-3)["sensor_xy"] for k in range(48)])
    assert np.ptp(hits, axis=0).max() > 100 * max(spreads) + 1.0


def test_sensor_turned_away_misses():
    rows = _ideal_lens(1.0, 0.1, 5e-3)
    opt = _optics(rows, 1.12, aim_z=1.0, aim_r=5e-3).tilt_sensor(0.0, math.pi)   # facing away
    st = oracle.trace(None, opt, [0.0, 0.0, 0.0], 1, 0, 0, 0, oracle.RK4, 1e-3)
    assert st["status"] == oracle.KILLED_MISS
