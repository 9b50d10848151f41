"""GPU parity of the simulated BOS experiment (Sec. 4) through the C ABI:
per-dot mean displacements and centroids (pivbos_bos_displacements), the
Eq. 9 theory along each dot's chief ray (pivbos_bos_theory) and the bilinear
regular-grid map (pivbos_regrid_bilinear), against the CPU FP64 oracle on the
same seeded inputs.  Positions and displacements: <= 1e-5 px; pair counts
exact; the grid map within its fixed-point error bound."""
import math

import numpy as np
import pytest

import oracle
from paper_1812_05902_gb300 import scenes
from gpu_helpers import TOL_PX, gpu_handles

pytestmark = pytest.mark.gpu


def _gpu_bos(fr, handles=None, dots=None):
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    med, opt = handles if handles is not None else gpu_handles(fr)
    src = fr.sources if dots is None else dots
    n = len(src)
    d = torch.tensor(src, dtype=torch.float64, device="cuda")
    cen = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    disp = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    P.pivbos_bos_displacements(med.h, opt.h, d, n, fr.rays_per_source, fr.seed, fr.frame_index, fr.integrator,
                               fr.step, cen, disp, cnt)
    th = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    P.pivbos_bos_theory(med.h, opt.h, d, n, th)
    P.pivbos_sync()
    return cen.cpu().numpy(), disp.cpu().numpy(), cnt.cpu().numpy(), th.cpu().numpy()


def _oracle_bos(fr, dot_ids=None):
    med = oracle.Medium.from_scene(fr.medium)
    opt = oracle.Optics.from_scene(fr.optics)
    cen, disp, cnt = oracle.bos_displacements(med, opt, fr.sources, fr.rays_per_source, fr.seed, fr.frame_index,
                                              fr.integrator, fr.step, dot_ids=dot_ids)
    sel = fr.sources if dot_ids is None else fr.sources[dot_ids]
    o = fr.optics
    th = oracle.eq9_displacements(med, sel, o.aim_z, o.magnification, o.n_object, o.pitch)
    return cen, disp, cnt, th


def _compare(g, o):
    cen_g, disp_g, cnt_g, th_g = g
    cen_o, disp_o, cnt_o, th_o = o
    np.testing.assert_array_equal(cnt_g, cnt_o)
    ok = cnt_o > 0
    assert np.isnan(cen_g[~ok]).all() and np.isnan(disp_g[~ok]).all()
    err = {"centroid": float(np.max(np.abs(cen_g[ok] - cen_o[ok]), initial=0.0)),
           "displacement": float(np.max(np.abs(disp_g[ok] - disp_o[ok]), initial=0.0)),
           "theory": float(np.max(np.abs(th_g - th_o), initial=0.0))}
    assert err["centroid"] <= TOL_PX, err
    assert err["displacement"] <= TOL_PX, err
    assert err["theory"] <= TOL_PX, err
    return err


@pytest.mark.parametrize("integ", [scenes.EULER, scenes.RK4])
def test_c0_slab_dots_match_oracle(integ):
    fr = scenes.c0(scale=0.01, rays_per_source=37)[0]     # 6 x 6 dots, ragged ray count
    fr.integrator = integ
    g = _gpu_bos(fr)
    o = _oracle_bos(fr)
    _compare(g, o)
    # Eq. 9 in the slab: the traced mean displacement equals the theory to
    # first order (checked on the oracle at 1.5e-3; the same holds here)
    np.testing.assert_allclose(g[1][:, 1], g[3][:, 1], rtol=2e-3)


def test_table1_small_grid_matches_oracle():
    fr = scenes.table1(scale=0.004, grid=64, rays_per_source=61)[0]   # 20 dots on a 64^2 slice
    g = _gpu_bos(fr)
    o = _oracle_bos(fr)
    err = _compare(g, o)
    assert (g[2] > 0).sum() >= 15
    assert np.abs(g[1][g[2] > 0]).max() > 0.05, err     # the field moves the dots


def test_displacements_are_bit_reproducible_and_edge_cases():
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    fr = scenes.table1(scale=0.01, grid=64, rays_per_source=200)[0]
    h = gpu_handles(fr)
    a = _gpu_bos(fr, h)
    b = _gpu_bos(fr, h)
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)
    # a dot whose image misses the sensor: no pairs, NaN
    far = np.array([[0.5, 0.5, 0.0]])
    cen, disp, cnt, th = _gpu_bos(fr, h, dots=far)
    assert cnt[0] == 0 and np.isnan(cen).all() and np.isnan(disp).all()
    # no dots, no rays: nothing to do / every dot without pairs
    med, opt = h
    empty = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    P.pivbos_bos_displacements(med.h, opt.h, empty, 0, 10, 0, 0, scenes.RK4, 1e-4)
    d = torch.tensor(fr.sources[:3], device="cuda")
    cnt = torch.full((3,), 7, dtype=torch.int32, device="cuda")
    P.pivbos_bos_displacements(med.h, opt.h, d, 3, 0, 0, 0, scenes.RK4, 1e-4, n_pairs=cnt)
    P.pivbos_sync()
    assert (cnt.cpu().numpy() == 0).all()


def test_theory_and_grid_edge_cases():
    """Eq. 9 is zero for a chief ray that misses the box or runs parallel to
    the sensor; an empty grid map is all NaN with zero weight."""
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    fr = scenes.c0(scale=0.01, rays_per_source=8)[0]
    med, opt = gpu_handles(fr)
    dots = torch.tensor([[0.2, 0.2, 0.0],                       # chief ray misses the box
                         [0.0, 0.0, fr.optics.aim_z],           # at the lens plane: no chief ray
                         [1e-3, 2e-3, 0.0]], dtype=torch.float64, device="cuda")
    th = torch.full((3, 2), 7.0, dtype=torch.float64, device="cuda")
    P.pivbos_bos_theory(med.h, opt.h, dots, 3, th)
    P.pivbos_sync()
    t = th.cpu().numpy()
    assert (t[:2] == 0.0).all() and abs(t[2, 1]) > 0.0
    out = torch.full((4, 5, 2), 3.0, dtype=torch.float64, device="cuda")
    w = torch.full((4, 5), 3.0, dtype=torch.float64, device="cuda")
    empty = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    P.pivbos_regrid_bilinear(empty, empty, 0, 5, 4, 0.0, 0.0, 1.0, 0.0, out, w)
    P.pivbos_sync()
    assert torch.isnan(out).all() and (w == 0.0).all()


def test_dot_ranges_reproduce_the_whole_set():
    """Dots split into ranges with global indices (one range per rank of a
    sharded run) give the whole set's results bit for bit."""
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    fr = scenes.table1(scale=0.004, grid=64, rays_per_source=97)[0]
    h = gpu_handles(fr)
    whole = _gpu_bos(fr, h)
    n = len(fr.sources)
    parts = []
    for first, count in ((0, 7), (7, n - 7)):
        d = torch.tensor(fr.sources[first:first + count], dtype=torch.float64, device="cuda")
        cen = torch.empty((count, 2), dtype=torch.float64, device="cuda")
        disp = torch.empty((count, 2), dtype=torch.float64, device="cuda")
        cnt = torch.empty(count, dtype=torch.int32, device="cuda")
        P.pivbos_bos_displacements_range(h[0].h, h[1].h, d, count, first, fr.rays_per_source, fr.seed,
                                         fr.frame_index, fr.integrator, fr.step, cen, disp, cnt)
        P.pivbos_sync()
        parts.append((cen.cpu().numpy(), disp.cpu().numpy(), cnt.cpu().numpy()))
    for k in range(3):
        assert np.array_equal(np.concatenate([p[k] for p in parts]), whole[k], equal_nan=True)


def test_full_size_table1_sampled_dots():
    """The bench's Table 1 workload at full size (5,120 dots x 1e4 rays, 256^2
    slice): sampled dots against the oracle, and Eq. 9 against the traced
    displacements over all dots (they agree up to the smoothing of each
    dot's ray cone, the effect the paper describes)."""
    fr = scenes.table1()[0]
    g = _gpu_bos(fr)
    ids = np.array([0, 1, 1777, 4095, 5119])
    o = _oracle_bos(fr, dot_ids=ids)
    _compare(tuple(x[ids] for x in g), o)
    cen, disp, cnt, th = g
    ok = cnt > 0.9 * fr.rays_per_source
    assert ok.sum() > 4000
    for c in range(2):
        r = np.corrcoef(disp[ok, c], th[ok, c])[0, 1]
        assert r > 0.9, (c, r)
        slope = np.sum(disp[ok, c] * th[ok, c]) / np.sum(th[ok, c] ** 2)
        assert 0.5 < slope < 1.0, (c, slope)


def test_regrid_matches_oracle():
    import torch
    from paper_1812_05902_gb300 import pivbos as P
    rng = np.random.default_rng(11)
    n = 3000
    xy = rng.uniform(-5.0, 520.0, (n, 2))
    vals = rng.normal(0.0, 1.5, (n, 2))
    vals[7] = np.nan                         # skipped
    W, H, x0, y0, cell = 33, 34, 0.0, -3.0, 16.0
    for min_w in (0.0, 0.05):
        out_o, w_o = oracle.regrid_bilinear(xy, vals, W, H, x0, y0, cell, min_weight=min_w)
        out = torch.empty((H, W, 2), dtype=torch.float64, device="cuda")
        w = torch.empty((H, W), dtype=torch.float64, device="cuda")
        P.pivbos_regrid_bilinear(torch.tensor(xy, device="cuda"), torch.tensor(vals, device="cuda"), n, W, H, x0,
                                 y0, cell, min_w, out, w)
        P.pivbos_sync()
        out_g, w_g = out.cpu().numpy(), w.cpu().numpy()
        np.testing.assert_allclose(w_g, w_o, rtol=0, atol=n * 2.0 ** -40)
        assert np.array_equal(np.isnan(out_g), np.isnan(out_o))
        keep = ~np.isnan(out_o[..., 0])
        # fixed-point bound: n 2^-32 (1 + |mean|) / weight
        bound = n * 2.0 ** -32 * (1.0 + np.abs(out_o[keep])) / w_o[keep][:, None] + 1e-12
        assert (np.abs(out_g[keep] - out_o[keep]) <= bound).all()
        firm = keep & (w_o >= 0.01)
        assert np.abs(out_g[firm] - out_o[firm]).max() < 1e-5
