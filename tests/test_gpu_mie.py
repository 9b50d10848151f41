"""GPU parity of the Mie radiance (Sec. 3.1) through the C ABI: the series
kernel's |S1|^2, |S2|^2 tables and efficiencies against the oracle, renders
whose rays carry the radiance (polarised and unpolarised laser) against the
oracle's weighted render, and the weighted deposit against the plain one
when every weight is 1."""
import math

import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes
from gpu_helpers import gpu_render

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,m_re,m_im", [(1e-6, 1.45, 0.0), (0.2e-6, 1.59, 0.0), (5e-6, 1.33, 0.0),
                                         (2e-6, 1.5, 0.05)])
def test_mie_tables_match_oracle(d, m_re, m_im):
    from paper_1812_05902_gb300 import pivbos as P
    n_med, lam = 1.000277, 532e-9
    g, qg = P.pivbos_mie(d, lam, n_med, m_re, m_im, 721)
    o, qo = oracle.mie(oracle.mie_size_parameter(d, lam, n_med), m_re, m_im, 721)
    np.testing.assert_allclose(g, o, rtol=1e-9, atol=1e-12 * o.max())
    for k in ("q_ext", "q_sca", "re_s0"):
        np.testing.assert_allclose(qg[k], qo[k], rtol=1e-10)
    assert qg["terms"] == qo["terms"]


def _weighted_frame(pol):
    fr = scenes.c1(scale=0.003)[0]                  # 30 particles x 300 rays
    fr.optics.mie = scenes.Mie(n_angles=1801, polarisation=pol)
    return fr


@pytest.mark.parametrize("pol", [(0.0, 1.0, 0.0), None], ids=["polarised", "unpolarised"])
def test_weighted_render_matches_oracle(pol):
    fr = _weighted_frame(pol)
    img_g, st_g = gpu_render(fr)
    img_o, st_o = oracle.render_frame(fr)
    assert np.array_equal(st_g, st_o)
    a, b = img_g.astype(np.float64), img_o.astype(np.float64)
    rel = math.sqrt(np.sum((a - b) ** 2)) / math.sqrt(np.sum(b * b))
    assert rel <= 1e-4, rel
    # each ray adds round(w 2^32): the totals agree to the FP32 weights
    np.testing.assert_allclose(img_g.sum(), img_o.sum(), rtol=2e-6)
    # the radiance matters: the weighted total is well below 2^32 per ray
    assert img_g.sum() < 0.9 * (int(st_g[0]) << 32)


def test_unit_weights_reproduce_the_plain_render():
    from paper_1812_05902_gb300 import pivbos as P
    import torch
    fr = scenes.c1(scale=0.003)[0]
    plain, st_p = gpu_render(fr)
    med = P.Medium(fr.medium)
    opt = P.Optics(fr.optics)
    ones = np.ones((64, 2))
    for pol in ((0.0, 1.0, 0.0), None):
        h = P.pivbos_optics_radiance(opt.h, (1.0, 0.0, 0.0), pol, ones)
        try:
            img = torch.zeros((fr.optics.height, fr.optics.width), dtype=torch.int64, device="cuda")
            src = torch.tensor(fr.sources, dtype=torch.float64, device="cuda")
            P.pivbos_render(med.h, h, src, len(fr.sources), fr.rays_per_source, fr.seed, fr.frame_index,
                            fr.integrator, fr.step, img)
            P.pivbos_sync()
            assert np.array_equal(img.cpu().numpy(), plain)
        finally:
            P.pivbos_optics_destroy(h)
