"""The seeded synthetic inputs follow the recipes the design states: the
k^-5/3 Gaussian random fields (spectral slope, mean, rms, no k = 0 mode),
the dissipation cutoff of the Table 1 slice, the shock and gradient
profiles, and the Table 1 geometry (dot density, magnification, distances)."""
import math

import numpy as np
import pytest

from paper_1812_05902_gb300 import scenes


def _radial_power(f):
    """Shell-averaged |f_hat|^2 against |k| (integer shells)."""
    F = np.fft.fftn(f - f.mean())
    P = np.abs(F) ** 2
    ks = np.meshgrid(*[np.fft.fftfreq(n) * n for n in f.shape], indexing="ij")
    k = np.sqrt(sum(x * x for x in ks))
    kb = np.rint(k).astype(int)
    num = np.bincount(kb.ravel(), P.ravel())
    cnt = np.bincount(kb.ravel())
    return np.arange(len(num)), num / np.maximum(cnt, 1)


def test_turbulence_field_spectrum_and_moments():
    rho = scenes.turbulence_rho(64, seed=2).astype(np.float64)
    assert abs(rho.mean() - 1.2) < 1e-6
    assert abs(rho.std() / 1.2 - 0.05) < 1e-5
    k, p = _radial_power(rho)
    sel = (k >= 3) & (k <= 20)
    slope = np.polyfit(np.log(k[sel]), np.log(p[sel]), 1)[0]
    # E(k) ~ k^-5/3 in 3-D: |rho_hat|^2 ~ k^-11/3
    assert abs(slope + 11.0 / 3.0) < 0.25, slope


def test_table1_slice_spectrum_with_cutoff():
    n, kc = 128, 8.0
    rho = scenes.turbulence_slice_rho(n, seed=5, mean=1.225, rms_frac=0.05, k_cut=kc)
    assert abs(rho.mean() - 1.225) < 1e-9
    assert abs(rho.std() / 1.225 - 0.05) < 1e-9
    k, p = _radial_power(rho)
    sel = (k >= 2) & (k <= 24)
    # 2-D: |rho_hat|^2 ~ k^-8/3 exp(-k^2 / k_cut^2)
    resid = np.log(p[sel]) + 8.0 / 3.0 * np.log(k[sel]) + k[sel] ** 2 / kc ** 2
    assert np.std(resid) < 0.35, np.std(resid)


def test_shock_and_gradient_profiles():
    rho = scenes.shock_rho(4, 201, 3, 1e-4, rho1=1.2, ratio=2.5, width=0.5e-3)
    y = np.arange(201) * 1e-4
    exp = 1.2 + 1.5 * 1.2 * 0.5 * (1.0 + np.tanh((y - 0.01) / 0.5e-3))
    np.testing.assert_allclose(rho[1, :, 2], exp, rtol=1e-6)
    g = scenes.linear_gradient_rho(5, 33, 4, 1.20, 1.26, axis=1)
    np.testing.assert_allclose(g[2, :, 3], np.linspace(1.20, 1.26, 33), rtol=1e-6)


def test_table1_geometry():
    t = scenes.TABLE1
    fr = scenes.table1()[0]
    o, m = fr.optics, fr.medium
    assert len(fr.sources) == 5120                       # 20 dots per 32 x 32 px on 512^2
    assert fr.rays_per_source == 10000
    np.testing.assert_allclose(o.magnification, t["f"] / (t["Z_A"] + t["Z_D"] - t["f"]))
    assert abs(o.magnification - t["M_printed"]) < 0.005
    # the lens sits Z_A + Z_D from the dots, the volume mid-plane Z_D
    np.testing.assert_allclose(o.aim_z, t["Z_A"] + t["Z_D"])
    z_mid = m.origin[2] + 0.5 * (m.dims[2] - 1) * m.spacing[2]
    np.testing.assert_allclose(z_mid, t["Z_D"])
    np.testing.assert_allclose(np.array(m.extent()) - np.array(m.origin), (t["Lx"], t["Ly"], t["Lz"]))
    # z-stacked: every depth layer is the same slice
    assert np.array_equal(m.rho[0], m.rho[-1])
    assert m.K == t["K"] and o.pitch == t["pitch"]
    # dots fill the field of view at the dot plane
    half = 0.5 * o.width * o.pitch / o.magnification
    assert np.abs(fr.sources[:, :2]).max() <= half and np.abs(fr.sources[:, :2]).max() > 0.95 * half
    assert (fr.sources[:, 2] == 0.0).all()


@pytest.mark.parametrize("scale", [1.0, 0.01])
def test_workload_sizes(scale):
    fr = scenes.c1(scale=scale)[0]
    assert len(fr.sources) == max(1, round(10000 * scale))
    c4 = scenes.c4(scale=scale, grid=32)[0]
    assert len(c4.sources) == max(1, round(100000 * scale))
    assert c4.rays_per_source == max(1, round(10000 * min(1.0, scale * 100)))
