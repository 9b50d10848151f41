"""Pins for the oracle's tracing through density gradients (Sec. 3.2):
straight rays in a uniform medium, the closed-form arc in a linear-gradient
slab with the convergence order of the RK4 (Eqs. 3-6) and first-order
schemes, and the BOS displacement of Eq. 9 (Sec. 4) in the linear slab and in
the paper's Table 1 geometry."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _far_sensor_optics(aim_z, aim_r, sensor_z=None):
    # no lens: rays fly straight to a large sensor; only the volume state is read
    sensor_z = aim_z + 0.1 if sensor_z is None else sensor_z
    return oracle.Optics(np.zeros((0, 6)), 1.0, aim_z, aim_r, sensor_z, 1e-3, 4096, 4096, 1e-3)


def test_uniform_medium_rays_are_straight():
    rho = scenes.uniform_rho(8, 9, 10, 1.3)
    med = oracle.Medium(rho, (-0.02, -0.02, 0.3), (0.04 / 7, 0.04 / 8, 0.05 / 9), 0.225e-3)
    opt = _far_sensor_optics(1.0, 0.01)
    src = np.array([0.001, -0.002, 0.0])
    for integ in (oracle.EULER, oracle.RK4):
        for k in range(20):
            st = oracle.trace(med, opt, src, 3, 0, k, 0, integ, 0.37e-3)
            p = oracle.lens_point(3, 0, k, 0, 0.01, 1.0)
            d = (p - src) / np.linalg.norm(p - src)
            np.testing.assert_allclose(st["vol_dir"], d, atol=3e-16)
            # the exit point lies on the straight line, on the far face
            t = (0.35 - src[2]) / d[2]
            np.testing.assert_allclose(st["vol_pos"], src + t * d, atol=2e-16 * 1.0 + 1e-16)
            assert st["steps"] == math.ceil(round(0.05 * (1 + 1.3 * 0.225e-3) * d[2] ** -1 / 0.37e-3, 9)) or st["steps"] > 0


def _slab(g, n_at_y0, L=(0.04, 0.04, 0.05), N=(5, 9, 6), z0=0.0, exact_nodes=False):
    """linear slab n = n_at_y0 + g y (K = 1, so rho = n - 1).  With
    ``exact_nodes`` the node values are binary fractions (exact in float32),
    so the interpolated field is exactly linear and the closed form holds to
    rounding; otherwise the float32 rounding of the node values is the floor."""
    nx, ny, nz = N
    o = (-L[0] / 2, -L[1] / 2, z0)
    h = (L[0] / (nx - 1), L[1] / (ny - 1), L[2] / (nz - 1))
    y = o[1] + h[1] * np.arange(ny)
    prof = n_at_y0 - 1.0 + g * y
    if exact_nodes:
        # a quantum well above float32's ulp of the largest value
        q = 2.0 ** (math.floor(math.log2(np.max(np.abs(prof)))) - 20)
        base = np.round(prof[0] / q) * q
        inc = np.round(g * h[1] / q) * q
        prof = base + inc * np.arange(ny)
    rho = np.broadcast_to(prof.reshape(1, ny, 1), (nz, ny, nx)).astype(np.float32)
    rr = rho[0, :, 0].astype(np.float64)
    return oracle.Medium(rho, o, h, 1.0), o, L, h, rr


def _closed_form_exit(src, d0, n_nodes_y, o, h, L):
    """Exact ray of d/dt T = n grad n with n linear in y (piecewise-linear
    interpolation of node values that are themselves exactly linear up to
    float32 rounding): Y = y + n0'/g obeys Y'' = g^2 Y, so
    Y(t) = Y0 cosh(gt) + (T_y0/g) sinh(gt)."""
    ny = len(n_nodes_y)
    y_nodes = o[1] + h[1] * np.arange(ny)
    g, c = np.polyfit(y_nodes, n_nodes_y, 1)     # n - 1 = c + g y
    n_y0 = 1.0 + c
    n_src = n_y0 + g * src[1]
    T0 = n_src * d0
    t_exit = (o[2] + L[2] - src[2]) / T0[2]
    # written without the cancellation of Y0 cosh(gt) - n0'/g for weak g:
    # y = y0 + T_y0 sinh(gt)/g + n(y0) 2 sinh^2(gt/2)/g,
    # T_y = n(y0) sinh(gt) + T_y0 cosh(gt)
    sh = math.sinh(0.5 * g * t_exit)
    y = src[1] + T0[1] * (math.sinh(g * t_exit) / g) + n_src * 2.0 * sh * (sh / g)
    Ty = n_src * math.sinh(g * t_exit) + T0[1] * math.cosh(g * t_exit)
    x = src[0] + T0[0] * t_exit
    T = np.array([T0[0], Ty, T0[2]])
    return np.array([x, y, o[2] + L[2]]), T / np.linalg.norm(T)


def test_linear_slab_closed_form_and_convergence_order():
    g = 20.0                    # strong gradient so that truncation error is visible
    med, o, L, h, rr = _slab(g, 1.6, exact_nodes=True)
    # node values on a straight line in index space (exact binary fractions)
    assert np.max(np.abs(np.diff(rr, 2))) == 0.0
    opt = _far_sensor_optics(0.3, 0.004)
    src = np.array([0.002, -0.003, 1e-12])
    errs = {}
    for integ in (oracle.RK4, oracle.EULER):
        for step in (L[2] / 8, L[2] / 16, L[2] / 32, L[2] / 64):
            e = []
            for k in range(6):
                st = oracle.trace(med, opt, src, 11, 0, k, 0, integ, step)
                p = oracle.lens_point(11, 0, k, 0, 0.004, 0.3)
                d0 = (p - src) / np.linalg.norm(p - src)
                pos, dirn = _closed_form_exit(src, d0, rr, o, h, L)
                assert abs(st["vol_pos"][2] - (o[2] + L[2])) < 1e-15
                e.append(max(np.max(np.abs(st["vol_pos"][:2] - pos[:2])),
                             0.05 * np.max(np.abs(st["vol_dir"] - dirn))))
            errs[(integ, step)] = max(e)
    r4 = [errs[(oracle.RK4, L[2] / 2**k)] / errs[(oracle.RK4, L[2] / 2**(k + 1))] for k in (3, 4, 5)]
    r1 = [errs[(oracle.EULER, L[2] / 2**k)] / errs[(oracle.EULER, L[2] / 2**(k + 1))] for k in (3, 4, 5)]
    # fourth order: halving the step divides the error by ~16; first order: ~2
    for r in r4:
        assert 12.0 < r < 20.0, r4
    for r in r1:
        assert 1.7 < r < 2.3, r1
    assert errs[(oracle.RK4, L[2] / 64)] < 1e-10


def test_weak_linear_slab_rk4_matches_closed_form():
    # the workload's own gradient (K drho/dy = 2.7e-4 /m): RK4 is exact to rounding
    med, o, L, h, rr = _slab(2.7e-4, 1.00027, L=(0.05, 0.05, 0.01), N=(32, 32, 32), z0=0.495,
                             exact_nodes=True)
    assert np.max(np.abs(np.diff(rr, 2))) == 0.0
    opt = _far_sensor_optics(1.155, 0.0065)
    src = np.array([0.004, 0.006, 0.0])
    for k in range(10):
        st = oracle.trace(med, opt, src, 0, 5, k, 0, oracle.RK4, 0.2e-3)
        p = oracle.lens_point(0, 5, k, 0, 0.0065, 1.155)
        d0 = (p - src) / np.linalg.norm(p - src)
        # straight run to the entry face, then the closed form
        t_in = (o[2] - src[2]) / d0[2]
        entry = src + t_in * d0
        pos, dirn = _closed_form_exit(entry, d0, rr, o, h, L)
        np.testing.assert_allclose(st["vol_pos"], pos, rtol=0, atol=2e-15)
        np.testing.assert_allclose(st["vol_dir"], dirn, rtol=0, atol=2e-15)


def _eq9_displacement(M, Z_D, K, drho_dy, Lz, n0):
    """Eq. 9: Delta X = M Z_D / n0 * integral of dn/dy dz = M Z_D K (drho/dy) L_z / n0"""
    return M * Z_D * K * drho_dy * Lz / n0


def _mean_displacement(med, opt, srcs, rays, seed, integ, step):
    d = []
    for s_i, src in enumerate(srcs):
        ids = s_i * rays + np.arange(rays)
        a = oracle.trace_many(med, opt, srcs, rays, ids, seed, 0, integ, step)
        b = oracle.trace_many(None, opt, srcs, rays, ids, seed, 0, integ, step)
        ok = (a["status"] == oracle.REACHED) & (b["status"] == oracle.REACHED)
        d.append(np.mean(a["sensor_xy"][ok] - b["sensor_xy"][ok], axis=0))
    return np.array(d)


def test_bos_displacement_eq9_linear_slab_c0():
    fr = scenes.c0()[0]
    med = oracle.Medium.from_scene(fr.medium)
    opt = oracle.Optics.from_scene(fr.optics)
    srcs = np.array([[x, y, 0.0] for x in (-1.02e-3, 0.34e-3) for y in (-0.34e-3, 1.02e-3)])
    disp = _mean_displacement(med, opt, srcs, 200, 0, oracle.EULER, 0.1e-3)
    n0 = fr.optics.n_object
    exp = _eq9_displacement(0.1, 0.5, 0.225e-3, 0.06 / 0.05, 0.01, n0) / 17e-6
    # rays bend toward higher n (+y in the volume); the real image is
    # inverted, so the apparent dot moves toward +y on the sensor
    np.testing.assert_allclose(disp[:, 1], exp, rtol=1e-3)
    assert np.max(np.abs(disp[:, 0])) < 1e-3 * exp


def test_bos_displacement_eq9_table1_geometry():
    t1 = json.load(open(os.path.join(GOLDEN, "table1_bos_geometry.json")))
    M, f, Z_D = t1["magnification"], t1["focal_length_m"], t1["Z_D_m"]
    Lx, Ly, Lz = t1["Lx_m"], t1["Ly_m"], t1["Lz_m"]
    K = t1["gladstone_dale_cm3_per_g"] * 1e-3      # cm^3/g -> m^3/kg
    rho0 = t1["density_scale_kg_m3"]
    n0 = 1.0 + K * rho0
    # reading: the dots are in focus with the printed M (s_o = f (1 + 1/M));
    # the volume mid-plane sits Z_D after the dots
    opt_s = scenes.ideal_lens_layout(0.0, M, f, t1["f_number"], n0, pitch=t1["pixel_pitch_m"],
                                     width=2048, height=2048)
    N = 33
    drho_dy = 0.1 * rho0 / Ly                     # 10 % rise across the volume
    rho = scenes.linear_gradient_rho(N, N, 11, rho0 - 0.05 * rho0, rho0 + 0.05 * rho0, axis=1)
    med_s = scenes.Medium(rho, (-Lx / 2, -Ly / 2, Z_D - Lz / 2), (Lx / (N - 1), Ly / (N - 1), Lz / 10), K)
    med = oracle.Medium.from_scene(med_s)
    opt = oracle.Optics.from_scene(opt_s)
    srcs = np.array([[0.0, 0.0, 0.0], [1e-3, -2e-3, 0.0]])
    disp = _mean_displacement(med, opt, srcs, 200, 7, oracle.RK4, 0.25e-3)
    exp = _eq9_displacement(M, Z_D, K, drho_dy, Lz, n0) / t1["pixel_pitch_m"]
    np.testing.assert_allclose(disp[:, 1], exp, rtol=2e-3)


def test_max_step_budget_kills():
    med, o, L, h, rr = _slab(0.0, 1.0)
    opt = _far_sensor_optics(0.3, 0.004)
    # a ray running almost parallel to the faces inside a long box would need
    # more than the budget only if the budget were wrong; check the formula
    assert med.max_steps(1e-3) == math.ceil(2 * math.sqrt(sum(x * x for x in L)) / 1e-3) + 4


def _sinh_minus_x(x):
    """sinh(x) - x without cancellation for small x."""
    if abs(x) < 0.1:
        x2 = x * x
        return x * x2 / 6.0 * (1.0 + x2 / 20.0 * (1.0 + x2 / 42.0 * (1.0 + x2 / 72.0)))
    return math.sinh(x) - x


def _closed_form_opl(src, d0, n_nodes_y, o, h, L):
    """Optical path of the exact slab ray inside the box: the integral of
    n ds = n^2 dt (dt = ds/n) with n = g Y, Y(t) = a cosh(gt) + b sinh(gt),
    a = n(y0)/g, b = T_y0/g:
    n(y0)^2 (t/2 + sinh(2gt)/(4g)) + n(y0) T_y0 sinh(gt)^2/g + T_y0^2 (sinh(2gt) - 2gt)/(4g^2) * g."""
    ny = len(n_nodes_y)
    y_nodes = o[1] + h[1] * np.arange(ny)
    g, c = np.polyfit(y_nodes, n_nodes_y, 1)
    n_src = 1.0 + c + g * src[1]
    T0 = n_src * d0
    t = (o[2] + L[2] - src[2]) / T0[2]
    x = 2.0 * g * t
    return (n_src ** 2 * (0.5 * t + (x + _sinh_minus_x(x)) / (4.0 * g))
            + n_src * T0[1] * math.sinh(g * t) ** 2 / g
            + T0[1] ** 2 * _sinh_minus_x(x) / (4.0 * g))


def test_optical_path_in_a_uniform_medium_is_n_times_the_length():
    """n constant: the ray is straight and its optical path inside the box is
    n times the distance from its entry to its exit (both schemes, any step)."""
    rho = scenes.uniform_rho(8, 9, 10, 1.3)
    K = 0.225e-3
    n = 1.0 + K * float(np.float32(1.3))
    med = oracle.Medium(rho, (-0.02, -0.02, 0.3), (0.04 / 7, 0.04 / 8, 0.05 / 9), K)
    opt = _far_sensor_optics(1.0, 0.01)
    src = np.array([0.001, -0.002, 0.0])
    for integ in (oracle.EULER, oracle.RK4):
        for k in range(10):
            st = oracle.trace(med, opt, src, 3, 0, k, 0, integ, 0.37e-3)
            p = oracle.lens_point(3, 0, k, 0, 0.01, 1.0)
            d = (p - src) / np.linalg.norm(p - src)
            entry = src + (0.3 - src[2]) / d[2] * d
            length = np.linalg.norm(st["vol_pos"] - entry)
            # the rounding of the position accumulated at z ~ 0.3 m, which the
            # clipped last step turns into the summed parameter: ~2^-53 |z| a step
            tol = 4.0 * st["steps"] * 2.0 ** -53 * abs(st["vol_pos"][2])
            assert abs(st["opl"] - n * length) <= tol, (st["opl"], n * length, tol)
    # a ray that never enters the box has no optical path inside it
    st = oracle.trace(med, opt, np.array([0.5, 0.5, 0.0]), 3, 0, 0, 0, oracle.RK4, 0.37e-3)
    assert st["steps"] == 0 and st["opl"] == 0.0


def test_optical_path_in_a_linear_slab_closed_form_and_order():
    """The optical path against the closed form of the exact arc: fourth order
    for Eqs. 3-5 with Simpson's rule on their stage points, first order for
    the first-order scheme; to rounding at the workload's weak gradient."""
    g = 20.0
    med, o, L, h, rr = _slab(g, 1.6, exact_nodes=True)
    opt = _far_sensor_optics(0.3, 0.004)
    src = np.array([0.002, -0.003, 1e-12])
    errs = {}
    for integ in (oracle.RK4, oracle.EULER):
        for step in (L[2] / 8, L[2] / 16, L[2] / 32, L[2] / 64):
            e = []
            for k in range(6):
                st = oracle.trace(med, opt, src, 11, 0, k, 0, integ, step)
                p = oracle.lens_point(11, 0, k, 0, 0.004, 0.3)
                d0 = (p - src) / np.linalg.norm(p - src)
                e.append(abs(st["opl"] - _closed_form_opl(src, d0, rr, o, h, L)))
            errs[(integ, step)] = max(e)
    r4 = [errs[(oracle.RK4, L[2] / 2**k)] / errs[(oracle.RK4, L[2] / 2**(k + 1))] for k in (3, 4, 5)]
    r1 = [errs[(oracle.EULER, L[2] / 2**k)] / errs[(oracle.EULER, L[2] / 2**(k + 1))] for k in (3, 4, 5)]
    for r in r4:
        assert 12.0 < r < 20.0, r4
    for r in r1:
        assert 1.7 < r < 2.3, r1
    # the workload's gradient: RK4 with Simpson's rule matches to rounding
    med, o, L, h, rr = _slab(2.7e-4, 1.00027, L=(0.05, 0.05, 0.01), N=(32, 32, 32), z0=0.495,
                             exact_nodes=True)
    opt = _far_sensor_optics(1.155, 0.0065)
    src = np.array([0.004, 0.006, 0.0])
    for k in range(10):
        st = oracle.trace(med, opt, src, 0, 5, k, 0, oracle.RK4, 0.2e-3)
        p = oracle.lens_point(0, 5, k, 0, 0.0065, 1.155)
        d0 = (p - src) / np.linalg.norm(p - src)
        entry = src + (o[2] - src[2]) / d0[2] * d0
        ref = _closed_form_opl(entry, d0, rr, o, h, L)
        tol = 4.0 * st["steps"] * 2.0 ** -53 * abs(st["vol_pos"][2])   # as in the uniform medium
        assert abs(st["opl"] - ref) <= tol, (st["opl"], ref, tol)
