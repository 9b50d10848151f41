"""Pins for the oracle's image-pair helpers: the second frame's particles
moved by a velocity field (explicit midpoint rule over trilinear samples),
and the 16-bit image (Sec. 3.4: ~1e4 rays per particle give a 16-bit
dynamic range).  Against closed forms: translation, the midpoint rule's
exact map for linear fields, its order on a rotation, clamping, and exact
integer counts (one or two counts per ray, half-up rounding, clipping)."""
import numpy as np
import pytest

import oracle

O = (-0.01, -0.02, 0.3)
H = (0.001, 0.0015, 0.002)
N = (21, 27, 11)          # nx, ny, nz


def _grid_points():
    nx, ny, nz = N
    x = O[0] + np.arange(nx) * H[0]
    y = O[1] + np.arange(ny) * H[1]
    z = O[2] + np.arange(nz) * H[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X, Y, Z], -1)            # [nz, ny, nx, 3]


def _linear_field(A, b):
    P = _grid_points()
    return (P @ np.asarray(A).T + np.asarray(b)).astype(np.float64)


def test_uniform_field_translates():
    U = np.array([1.5, -0.25, 0.75])
    vel = np.broadcast_to(U, N[::-1] + (3,)).astype(np.float32)
    U32 = vel[0, 0, 0].astype(np.float64)
    rng = np.random.default_rng(2)
    src = np.array(O) + rng.random((50, 3)) * np.array(H) * (np.array(N) - 1)
    dt = 1e-3
    out = oracle.advect(src, vel, O, H, dt)
    np.testing.assert_allclose(out, src + dt * U32, rtol=0, atol=1e-15)
    # outside the grid the field is clamped to the nearest face: still a translation
    far = np.array([[0.5, 0.5, 0.0], [-1.0, 0.0, 2.0]])
    np.testing.assert_allclose(oracle.advect(far, vel, O, H, dt), far + dt * U32, rtol=0, atol=1e-15)


def test_linear_field_midpoint_map_exact():
    """For u = A x + b the midpoint rule maps x to
    (I + dt A + dt^2 A^2 / 2) x + dt (I + dt A / 2) b."""
    rng = np.random.default_rng(5)
    A = rng.normal(size=(3, 3)) * 20.0
    b = rng.normal(size=3) * 0.5
    vel64 = _linear_field(A, b)
    vel = vel64.astype(np.float32)
    # the float32 node values are the field the oracle interpolates: refit
    # A, b to them so the closed form uses the same linear field
    P = _grid_points().reshape(-1, 3)
    X = np.hstack([P, np.ones((len(P), 1))])
    coef, *_ = np.linalg.lstsq(X, vel.reshape(-1, 3).astype(np.float64), rcond=None)
    A32, b32 = coef[:3].T, coef[3]
    src = np.array(O) + (0.25 + 0.5 * rng.random((40, 3))) * np.array(H) * (np.array(N) - 1)
    dt = 1e-4
    out = oracle.advect(src, vel, O, H, dt)
    I = np.eye(3)
    M = I + dt * A32 + 0.5 * dt * dt * A32 @ A32
    exp = src @ M.T + dt * (I + 0.5 * dt * A32) @ b32
    np.testing.assert_allclose(out, exp, rtol=0, atol=2e-10)
    # the quadratic term matters: a first-order step misses it by far more
    euler = src + dt * (src @ A32.T + b32)
    assert np.abs(euler - exp).max() > 100 * np.abs(out - exp).max()


def test_second_order_on_a_rotation():
    w = 400.0
    A = np.array([[0.0, -w, 0.0], [w, 0.0, 0.0], [0.0, 0.0, 0.0]])
    vel = _linear_field(A, np.zeros(3)).astype(np.float32)
    x0 = np.array([[0.002, -0.004, 0.31]])

    def exact(dt):
        c, s = np.cos(w * dt), np.sin(w * dt)
        x, y, z = x0[0]
        return np.array([c * x - s * y, s * x + c * y, z])

    errs = [np.abs(oracle.advect(x0, vel, O, H, dt)[0] - exact(dt)).max() for dt in (2e-4, 1e-4)]
    # local error of the midpoint rule is third order in dt
    assert 6.0 < errs[0] / errs[1] < 10.0


def test_u16_conversion_exact():
    two32 = 1 << 32
    # full scale 65535 rays: one count per ray (d = 2^32 exactly)
    k = np.array([0, 1, 7, 1000, 65535, 65536, 200000], dtype=np.int64)
    assert oracle.image_u16(k * two32, 65535.0).tolist() == [0, 1, 7, 1000, 65535, 65535, 65535]
    # half the full scale: two counts per ray (d = 2^31)
    assert oracle.image_u16(k[:4] * two32, 65535.0 / 2).tolist() == [0, 2, 14, 2000]
    # rounding half up at the count boundaries, negatives clip to 0
    d = two32
    v = np.array([3 * d + d // 2 - 1, 3 * d + d // 2, 3 * d + d // 2 + 1, -5 * d], dtype=np.int64)
    assert oracle.image_u16(v, 65535.0).tolist() == [3, 4, 4, 0]
    # a full scale of 100 rays: counts = k * 655.35 rounded
    k = np.arange(0, 101, dtype=np.int64)
    assert np.array_equal(oracle.image_u16(k * two32, 100.0).astype(np.int64),
                          np.floor(k * 655.35 + 0.5).astype(np.int64))
