"""Pins for the oracle's sensor deposit (Sec. 3.4, Eq. 8): exact total
intensity, symmetry, the sigma -> 0 limit, pixel integrals of the Gaussian
against numerical quadrature, the spot width that Eq. 8 sets, and clipping
at the sensor edge."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1812_05902_gb300 import scenes

TWO32 = 2**32


def _opt(W=64, H=48, pitch=10e-6, sigma=12e-6):
    return oracle.Optics(np.zeros((0, 6)), 1.0, 1.0, 0.01, 2.0, pitch, W, H, sigma)


def test_each_ray_adds_exactly_two_to_the_32():
    rng = np.random.default_rng(0)
    opt = _opt()
    img = np.zeros((48, 64), dtype=np.int64)
    n = 500
    for _ in range(n):
        oracle.deposit(opt, rng.uniform(0, 64), rng.uniform(0, 48), img)
    assert img.sum() == n * TWO32
    assert img.min() >= 0


def test_render_total_equals_rays_reaching_sensor():
    fr = scenes.c0(scale=0.05, rays_per_source=20)[0]
    img, st = oracle.render_frame(fr)
    assert st.sum() == fr.n_rays
    assert img.sum() == st[oracle.REACHED] * TWO32


def test_centre_hit_is_symmetric():
    opt = _opt(sigma=17e-6)
    img = oracle.deposit(opt, 20.5, 10.5)
    nz = np.argwhere(img)
    j0, j1, i0, i1 = nz[:, 0].min(), nz[:, 0].max(), nz[:, 1].min(), nz[:, 1].max()
    win = img[j0:j1 + 1, i0:i1 + 1]
    assert win.shape == (11, 11)        # floor(p -+ 3 sigma): pixels 15..25 with sigma = 1.7 px
    # mirror symmetry in both axes and transposition (the remainder lands on
    # the central pixel, which is its own mirror image)
    assert np.array_equal(win, win[::-1, :])
    assert np.array_equal(win, win[:, ::-1])
    assert np.array_equal(win, win.T)
    assert win[5, 5] == win.max()


def test_small_sigma_puts_everything_in_one_pixel():
    opt = _opt(sigma=1e-9)
    img = oracle.deposit(opt, 7.3, 9.9)
    assert img[9, 7] == TWO32
    assert img.sum() == TWO32


@pytest.mark.parametrize("px,py,sigma_px", [(10.3, 20.71, 0.6), (33.02, 5.5, 1.3), (0.2, 47.9, 0.9)])
def test_pixel_weights_match_quadrature(px, py, sigma_px):
    pitch = 10e-6
    opt = _opt(pitch=pitch, sigma=sigma_px * pitch)
    img = oracle.deposit(opt, px, py)
    s = sigma_px
    pdf = lambda u, m: math.exp(-0.5 * ((u - m) / s) ** 2) / (s * math.sqrt(2 * math.pi))

    def weights(p, N):
        lo = max(int(math.floor(p - 3 * s)), 0)
        hi = min(int(math.floor(p + 3 * s)), N - 1)
        w = np.array([integrate.quad(pdf, i, i + 1, args=(p,), epsabs=1e-15, epsrel=1e-13)[0]
                      for i in range(lo, hi + 1)])
        return lo, w / w.sum()

    xlo, wx = weights(px, 64)
    ylo, wy = weights(py, 48)
    exp = np.zeros_like(img, dtype=np.float64)
    exp[ylo:ylo + len(wy), xlo:xlo + len(wx)] = np.outer(wy, wx) * TWO32
    diff = img - np.rint(exp)
    # everything except the remainder pixel agrees to rounding; the remainder
    # is at most half a unit per pixel
    jm, im = np.unravel_index(np.argmax(exp), exp.shape)
    mask = np.ones_like(diff, dtype=bool)
    mask[jm, im] = False
    assert np.max(np.abs(diff[mask])) <= 1
    assert abs(diff[jm, im]) <= 0.5 * len(wx) * len(wy) + 1


def test_spot_width_follows_eq8():
    # Eq. 8 sets d_tau; sigma = d_tau / 4.  A spot several pixels wide has
    # second moment sigma^2 (truncated at 3 sigma) plus the 1/12 px^2 of the
    # pixel box.
    f_number, M, lam = 8.0, 0.1, 532e-9
    for rule, factor in ((0, math.pi), (1, 1.0)):
        sigma = oracle.sigma_eq8(f_number, M, lam, rule)
        pitch = sigma / 3.0          # about three pixels per sigma
        opt = oracle.Optics(np.zeros((0, 6)), 1.0, 1.0, 0.01, 2.0, pitch, 64, 64, sigma)
        img = oracle.deposit(opt, 32.0, 32.0).astype(np.float64)
        prof = img.sum(axis=0) / img.sum()
        c = np.arange(64) + 0.5
        var = np.sum(prof * (c - 32.0) ** 2)
        s = sigma / pitch
        # variance of a Gaussian truncated at +-3 sigma
        a = 3.0
        trunc = 1.0 - 2 * a * math.exp(-a * a / 2) / (math.sqrt(2 * math.pi) * math.erf(a / math.sqrt(2)))
        assert abs(var - (s * s * trunc + 1.0 / 12.0)) < 0.03 * s * s
        d_tau = 4 * sigma
        assert abs(d_tau / (2.44 * f_number * (M + 1) * lam) - factor) < 1e-12


def test_edge_clipping_keeps_the_total():
    opt = _opt(sigma=20e-6)
    for px, py in ((0.01, 0.02), (63.99, 47.99), (0.5, 47.5)):
        img = oracle.deposit(opt, px, py)
        assert img.sum() == TWO32
        assert img.min() >= 0
