"""Pins for the oracle's medium (Sec. 3.2): Eq. 1 at the nodes, the node
gradient (exact on quadratics for the second-order differences used), and
trilinear sampling (exact on trilinear functions, clamped outside the box)."""
import numpy as np
import pytest

import oracle


def _grid(nx, ny, nz, h, origin):
    x = origin[0] + h[0] * np.arange(nx)
    y = origin[1] + h[1] * np.arange(ny)
    z = origin[2] + h[2] * np.arange(nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def test_gladstone_dale_at_nodes():
    rng = np.random.default_rng(0)
    rho = rng.uniform(0.5, 3.0, (5, 6, 7)).astype(np.float32)
    K = 0.226e-3
    m = oracle.Medium(rho, (0, 0, 0), (1e-3, 2e-3, 3e-3), K)
    dn, *_ = m.nodes()
    np.testing.assert_allclose(dn, K * rho.astype(np.float64), rtol=1e-15, atol=0)


@pytest.mark.parametrize("dims", [(7, 6, 5), (3, 4, 9)])
def test_gradient_exact_for_quadratic_density(dims):
    nx, ny, nz = dims
    h = (1.5e-3, 0.7e-3, 2.1e-3)
    o = (-0.01, 0.003, 0.2)
    X, Y, Z = _grid(nx, ny, nz, h, o)
    # quadratic in every variable, with cross terms; values are exactly
    # representable after the float32 cast only approximately, so the
    # expectation is computed from the float32 field by exact differences
    c = dict(a=1.2, bx=3.0, by=-2.0, bz=1.5, cx=40.0, cy=-25.0, cz=60.0, exy=11.0, eyz=-7.0)
    rho64 = (c["a"] + c["bx"] * X + c["by"] * Y + c["bz"] * Z + c["cx"] * X**2 + c["cy"] * Y**2
             + c["cz"] * Z**2 + c["exy"] * X * Y + c["eyz"] * Y * Z)
    rho = rho64.astype(np.float32)
    K = 0.225e-3
    m = oracle.Medium(rho, o, h, K)
    _, gx, gy, gz = m.nodes()
    # analytic derivative of the quadratic, times K
    ex = K * (c["bx"] + 2 * c["cx"] * X + c["exy"] * Y)
    ey = K * (c["by"] + 2 * c["cy"] * Y + c["exy"] * X + c["eyz"] * Z)
    ez = K * (c["bz"] + 2 * c["cz"] * Z + c["eyz"] * Y)
    # only the float32 rounding of rho remains: the one-sided formula weighs
    # the node errors by (3 + 4 + 1) / (2h) = 4/h, the central one by 1/h
    r_err = np.max(np.abs(rho.astype(np.float64) - rho64))
    for got, exp, hh in ((gx, ex, h[0]), (gy, ey, h[1]), (gz, ez, h[2])):
        assert np.max(np.abs(got - exp)) <= K * 4.0 * r_err / hh * 1.001 + 1e-18


def test_gradient_two_node_axis_uses_two_point_difference():
    rho = np.tile(np.array([1.0, 3.0], dtype=np.float32), (2, 2, 1))  # [nz=2, ny=2, nx=2]
    m = oracle.Medium(rho, (0, 0, 0), (0.5, 1.0, 1.0), 1.0)
    _, gx, gy, gz = m.nodes()
    np.testing.assert_allclose(gx, 4.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(gy, 0.0, atol=0)
    np.testing.assert_allclose(gz, 0.0, atol=0)


def test_trilinear_exact_on_trilinear_functions_and_clamped():
    nx, ny, nz = 6, 5, 4
    h = (1e-3, 2e-3, 0.5e-3)
    o = (0.01, -0.02, 0.3)
    X, Y, Z = _grid(nx, ny, nz, h, o)
    u, v, w = (X - o[0]) / h[0], (Y - o[1]) / h[1], (Z - o[2]) / h[2]
    f = lambda u, v, w: 1.0 + 0.3 * u - 0.2 * v + 0.1 * w + 0.05 * u * v - 0.07 * v * w + 0.02 * u * w + 0.01 * u * v * w
    rho = f(u, v, w).astype(np.float32)
    K = 1.0
    m = oracle.Medium(rho, o, h, K)
    rng = np.random.default_rng(1)
    pts = np.stack([o[a] + rng.uniform(-0.5, (n - 1) + 0.5, 400) * h[a]
                    for a, n in enumerate((nx, ny, nz))], axis=1)
    dn, g = m.sample(pts)
    # brute force: trilinear interpolation of the node values is the
    # trilinear function itself, evaluated at the clamped coordinates
    uu = np.clip((pts[:, 0] - o[0]) / h[0], 0, nx - 1)
    vv = np.clip((pts[:, 1] - o[1]) / h[1], 0, ny - 1)
    ww = np.clip((pts[:, 2] - o[2]) / h[2], 0, nz - 1)
    # the node values were rounded to float32, so compare against the
    # float32 node data interpolated by an independent brute-force routine
    r32 = rho.astype(np.float64)

    def brute(a, b, c):
        i = min(int(np.floor(a)), nx - 2); j = min(int(np.floor(b)), ny - 2); k = min(int(np.floor(c)), nz - 2)
        fa, fb, fc = a - i, b - j, c - k
        s = 0.0
        for di in (0, 1):
            for dj in (0, 1):
                for dk in (0, 1):
                    wgt = (fa if di else 1 - fa) * (fb if dj else 1 - fb) * (fc if dk else 1 - fc)
                    s += wgt * r32[k + dk, j + dj, i + di]
        return s

    exp = np.array([brute(a, b, c) for a, b, c in zip(uu, vv, ww)])
    np.testing.assert_allclose(dn, K * exp, rtol=0, atol=1e-14)
    # and against the analytic trilinear function (float32 rounding only)
    np.testing.assert_allclose(dn, f(uu, vv, ww), rtol=0, atol=5e-7)
