"""Pins for the oracle's simulated BOS experiment (Sec. 4): the depth
integral of the transverse gradient of n that Eq. 9 needs, the per-dot mean
displacement of the traced rays, and the bilinear regular-grid map the paper
draws the displacements on.  Each pin is something the oracle does not
compute itself: a closed form, a library routine (numpy.gradient,
scipy.ndimage.map_coordinates), brute force or a symmetry."""
import math

import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes

K = 0.225e-3


def _linear_slab(N=33, Lz=0.01, zc=0.5, axis=1):
    # rho = 1 + j/32 along y: every node value is exact in float32
    ramp = 1.0 + np.arange(N) / 32.0
    shape = [1, 1, 1]
    shape[2 - axis] = N
    rho = np.ascontiguousarray(np.broadcast_to(ramp.reshape(shape), (N, N, N)), dtype=np.float32)
    L = 0.032
    h = (L / (N - 1), L / (N - 1), Lz / (N - 1))
    origin = (-L / 2, -L / 2, zc - Lz / 2)
    g = K * (1.0 / 32.0) / h[axis]          # dn/dy
    return oracle.Medium(rho, origin, h, K), g, origin, h


def test_line_integral_linear_field_closed_form():
    med, g, origin, h = _linear_slab()
    Lz = 32 * h[2]
    # chief rays from dots 0.5 m before the mid-plane toward the lens centre
    for s in ((0.0, 0.0, 0.0), (3e-3, -4e-3, 0.0), (-11e-3, 9e-3, 0.01)):
        I, pieces = oracle.line_gradient_integral(med, s, (0.0, 0.0, 1.2))
        assert pieces >= 32
        np.testing.assert_allclose(I[1], g * Lz, rtol=1e-13)
        assert abs(I[0]) < 1e-12 * g * Lz


def test_line_integral_partial_crossing_and_miss():
    med, g, origin, h = _linear_slab()
    zlo = origin[2]
    # a line leaving through the +x face: only its part inside the box counts
    s = (0.0155, 0.0, zlo - 0.001)
    c = (0.0155 + 0.2, 0.0, zlo - 0.001 + 0.2 / 0.5)      # dx/dz = 0.5
    I, _ = oracle.line_gradient_integral(med, s, c)
    z_exit = s[2] + (0.016 - s[0]) / 0.5
    np.testing.assert_allclose(I[1], g * (z_exit - zlo), rtol=1e-12)
    # a line that misses the box
    I, k = oracle.line_gradient_integral(med, (0.05, 0.0, 0.0), (0.05, 0.0, 1.0))
    assert k == 0 and I[0] == 0.0 and I[1] == 0.0
    # the integral stops at the end point c inside the box
    I, _ = oracle.line_gradient_integral(med, (0.0, 0.0, 0.0), (0.0, 0.0, 0.5))
    np.testing.assert_allclose(I[1], g * (0.5 - zlo), rtol=1e-12)


def _random_field(seed=5, dims=(7, 6, 5)):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    rho = (1.2 + 0.3 * rng.standard_normal((nz, ny, nx))).astype(np.float32)
    origin = (-0.004, -0.003, 0.2)
    h = (0.0013, 0.0011, 0.0017)
    return rho, origin, h


def _library_node_gradients(rho, h):
    """numpy.gradient with second-order edges: the node gradient of Eq. 6's
    grid (central inside, one-sided second order at the faces)."""
    dn = K * rho.astype(np.float64)
    gz, gy, gx = np.gradient(dn, h[2], h[1], h[0], edge_order=2)
    return gx, gy


def test_line_integral_axis_parallel_is_trapezoid_of_node_column():
    rho, origin, h = _random_field()
    med = oracle.Medium(rho, origin, h, K)
    gx, gy = _library_node_gradients(rho, h)
    i, j = 3, 2
    x = origin[0] + i * h[0]
    y = origin[1] + j * h[1]
    I, _ = oracle.line_gradient_integral(med, (x, y, 0.0), (x, y, 1.0))
    # along a node column the trilinear sample is linear between nodes
    np.testing.assert_allclose(I[0], np.trapezoid(gx[:, j, i], dx=h[2]), rtol=1e-12)
    np.testing.assert_allclose(I[1], np.trapezoid(gy[:, j, i], dx=h[2]), rtol=1e-12)


def test_line_integral_oblique_against_dense_library_quadrature():
    from scipy.ndimage import map_coordinates
    rho, origin, h = _random_field()
    med = oracle.Medium(rho, origin, h, K)
    gx, gy = _library_node_gradients(rho, h)
    s = np.array([-0.0031, 0.0042, 0.17])
    c = np.array([0.0025, -0.0024, 0.23])
    I, pieces = oracle.line_gradient_integral(med, s, c)
    assert pieces >= 5
    # dense trapezoid over the part of the line inside the box, sampled by
    # scipy's linear spline (order 1 = trilinear)
    zlo, zhi = origin[2], origin[2] + 4 * h[2]
    ax = (c[:2] - s[:2]) / (c[2] - s[2])
    z = np.linspace(zlo, zhi, 400001)
    pts = s[:2][None, :] + (z - s[2])[:, None] * ax[None, :]
    inside = ((pts[:, 0] >= origin[0]) & (pts[:, 0] <= origin[0] + 6 * h[0]) &
              (pts[:, 1] >= origin[1]) & (pts[:, 1] <= origin[1] + 5 * h[1]))
    assert inside.all()   # this line crosses the box through both z faces
    coords = np.stack([(z - origin[2]) / h[2], (pts[:, 1] - origin[1]) / h[1], (pts[:, 0] - origin[0]) / h[0]])
    fx = map_coordinates(gx, coords, order=1, mode="nearest")
    fy = map_coordinates(gy, coords, order=1, mode="nearest")
    np.testing.assert_allclose(I, [np.trapezoid(fx, z), np.trapezoid(fy, z)], rtol=2e-8)


def test_eq9_theory_matches_traced_mean_displacement_in_a_slab():
    """The traced per-dot mean displacement and Eq. 9 agree for a linear slab
    (the bend happens at the mid-plane to first order)."""
    fr = scenes.c0()[0]
    med = oracle.Medium.from_scene(fr.medium)
    opt = oracle.Optics.from_scene(fr.optics)
    o = fr.optics
    dots = np.array([[-1.02e-3, 0.34e-3, 0.0], [0.34e-3, -1.02e-3, 0.0], [2.0e-3, 2.0e-3, 0.0]])
    cen, disp, cnt = oracle.bos_displacements(med, opt, dots, 200, 0, 0, oracle.EULER, 0.1e-3)
    th = oracle.eq9_displacements(med, dots, o.aim_z, o.magnification, o.n_object, o.pitch)
    assert (cnt == 200).all()
    np.testing.assert_allclose(disp[:, 1], th[:, 1], rtol=1.5e-3)
    assert np.abs(th[:, 0]).max() < 1e-9
    assert np.abs(disp[:, 0]).max() < 1e-3 * np.abs(disp[:, 1]).max()


def test_bos_displacement_zero_in_uniform_medium_and_centroid_is_the_image():
    """A uniform medium bends nothing; through the ideal lens every ray of a
    dot meets at its geometric image -(s_i/s_o) h (in pixels, no flip)."""
    fr = scenes.c0()[0]
    m = fr.medium
    med = oracle.Medium(scenes.uniform_rho(*m.dims, rho=1.2), m.origin, m.spacing, m.K)
    opt = oracle.Optics.from_scene(fr.optics)
    o = fr.optics
    dots = np.array([[1.5e-3, -0.7e-3, 0.0], [-4e-3, 2e-3, 0.0]])
    cen, disp, cnt = oracle.bos_displacements(med, opt, dots, 64, 9, 0, oracle.RK4, 0.2e-3)
    assert (cnt == 64).all()
    assert np.abs(disp).max() < 1e-9
    s_o = o.aim_z
    s_i = o.sensor_z - o.aim_z
    img = -(s_i / s_o) * dots[:, :2] / o.pitch + np.array([o.width / 2, o.height / 2])
    np.testing.assert_allclose(cen, img, atol=1e-8)


def test_bos_displacement_counts_only_pairs():
    fr = scenes.c0()[0]
    med = oracle.Medium.from_scene(fr.medium)
    # a sensor so small that the dot's image sits off it: no pairs, NaN
    o = fr.optics
    opt = oracle.Optics(o.surface_array(), o.n_object, o.aim_z, o.aim_r, o.sensor_z, o.pitch, 8, 8,
                        oracle.sigma_eq8(o.f_number, o.magnification, o.wavelength, o.dtau_rule))
    cen, disp, cnt = oracle.bos_displacements(med, opt, np.array([[5e-3, 5e-3, 0.0]]), 16, 0, 0,
                                              oracle.EULER, 0.1e-3)
    assert cnt[0] == 0 and np.isnan(cen).all() and np.isnan(disp).all()


def test_regrid_constant_and_single_point_weights():
    rng = np.random.default_rng(3)
    xy = rng.uniform(0.0, 40.0, (500, 2))
    vals = np.tile([0.25, -1.5], (500, 1))
    out, w = oracle.regrid_bilinear(xy, vals, 6, 6, 0.0, 0.0, 8.0)
    ok = w > 0
    assert ok.all()
    np.testing.assert_allclose(out[ok], np.tile([0.25, -1.5], (ok.sum(), 1)), rtol=1e-14)
    np.testing.assert_allclose(w.sum(), 500.0, rtol=1e-13)   # each point spreads unit weight
    # one point at (u, v) = (1.25, 2.5): weights (1-fu)(1-fv) ... on its cell
    out, w = oracle.regrid_bilinear([[10.0, 20.0]], [[2.0, 3.0]], 4, 4, 0.0, 0.0, 8.0)
    exp = np.zeros((4, 4))
    exp[2, 1], exp[2, 2], exp[3, 1], exp[3, 2] = 0.75 * 0.5, 0.25 * 0.5, 0.75 * 0.5, 0.25 * 0.5
    np.testing.assert_allclose(w, exp, rtol=1e-15)
    assert np.isnan(out[0, 0]).all()
    np.testing.assert_allclose(out[2, 1], [2.0, 3.0], rtol=1e-15)
    # a point on the far corner node belongs to the last cell
    out, w = oracle.regrid_bilinear([[24.0, 24.0]], [[1.0, 1.0]], 4, 4, 0.0, 0.0, 8.0)
    assert w[3, 3] == 1.0 and w.sum() == 1.0
    # outside the grid: ignored
    out, w = oracle.regrid_bilinear([[-0.5, 3.0], [3.0, 24.5]], [[1.0, 1.0], [1.0, 1.0]], 4, 4, 0.0, 0.0, 8.0)
    assert w.sum() == 0.0 and np.isnan(out).all()


def test_regrid_reproduces_linear_field_from_symmetric_points():
    """Points at the centres of every cell: an interior node receives four
    points placed symmetrically around it with weight 1/4 each, so a linear
    field comes back exactly at the interior nodes."""
    W, H, cell = 7, 6, 4.0
    cx = (np.arange(W - 1) + 0.5) * cell + 1.0
    cy = (np.arange(H - 1) + 0.5) * cell - 2.0
    X, Y = np.meshgrid(cx, cy)
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    f = lambda x, y: np.stack([0.3 + 0.01 * x - 0.02 * y, -1.0 + 0.05 * y], -1)
    out, w = oracle.regrid_bilinear(xy, f(xy[:, 0], xy[:, 1]), W, H, 1.0, -2.0, cell)
    nx = 1.0 + np.arange(W) * cell
    ny = -2.0 + np.arange(H) * cell
    NX, NY = np.meshgrid(nx, ny)
    exp = f(NX, NY)
    np.testing.assert_allclose(out[1:-1, 1:-1], exp[1:-1, 1:-1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(w[1:-1, 1:-1], 1.0, rtol=1e-15)
