"""The surrogate's per-bin plan (host code of pivbos_surrogate_train, through
the testing library's pivbos_plan_bins; no GPU): for each entry bin, the
projection alone, the projection with the network's correction, or the plain
fallback, at the least render cost whose served squared error stays within
the budget.  Checked on seeded synthetic bins: the budget holds, ineligible
bins fall back, the network is left out when asked, the returned cost is the
cost of the returned assignment, no plan costs more than falling back
everywhere, more budget never costs more, and the two limits (no budget,
unlimited budget) give the plans they must."""
import numpy as np
import pytest

SEGMENTS = 8
FB_FIXED = 7.0                          # plain steps of a fallback ray besides its integration steps
PROJ = 3.9 + 0.68 * SEGMENTS            # plain steps of a ray served by the projection
NET_EXTRA = 5.3                         # ... and by the network's correction on top


@pytest.fixture(scope="module")
def P():
    from paper_1812_05902_gb300 import pivbos as P
    try:
        P.testing_lib()
    except Exception as e:                   # pragma: no cover - the library must be built
        pytest.fail("testing library: %s" % e)
    return P


def _bins(seed, n=256):
    rng = np.random.default_rng(seed)
    cnt = rng.integers(0, 60, n)
    cnt[rng.random(n) < 0.1] = 0
    steps = cnt * rng.uniform(2.0, 150.0, n)
    err2p = cnt * rng.uniform(0.0, 1e-4, n) ** 2 * rng.uniform(0.0, 4.0, n)
    err2n = err2p * rng.uniform(0.1, 1.2, n)
    return err2n, err2p, steps, cnt


def _cost(served, network, steps, cnt):
    fb = ~served
    return float(np.sum((steps + FB_FIXED * cnt)[fb]) + np.sum(PROJ * cnt[served & ~network]) +
                 np.sum((PROJ + NET_EXTRA) * cnt[served & network]))


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("with_net", [True, False])
def test_plan_respects_budget_and_eligibility_and_prices_itself(P, seed, with_net):
    err2n, err2p, steps, cnt = _bins(seed)
    min_count = 5
    total2 = float(np.sum(err2p))
    for frac in (0.0, 0.05, 0.3, 1.0):
        budget2 = frac * total2
        served, network, m = P.pivbos_plan_bins(err2n, err2p, steps, cnt, min_count, budget2, SEGMENTS, with_net)
        err = np.where(network, err2n, err2p)
        # the budget, the summaries
        assert m["err2"] <= budget2 * (1 + 1e-12) + 1e-300
        assert np.isclose(m["err2"], np.sum(err[served]), rtol=1e-12, atol=1e-300)
        assert m["rays"] == np.sum(cnt[served]) and m["net_rays"] == np.sum(cnt[network])
        assert np.isclose(m["steps"], np.sum(steps[served]), rtol=1e-12)
        # eligibility; the network only where allowed and only on served bins
        assert not np.any(served & (cnt < min_count))
        assert not np.any(network & ~served)
        if not with_net:
            assert not np.any(network)
        # the returned cost is the assignment's cost, never above falling back everywhere
        assert np.isclose(m["cost"], _cost(served, network, steps, cnt), rtol=1e-9)
        assert m["cost"] <= float(np.sum(steps + FB_FIXED * cnt)) * (1 + 1e-12)


@pytest.mark.parametrize("seed", [5, 6])
def test_more_budget_never_costs_more(P, seed):
    err2n, err2p, steps, cnt = _bins(seed)
    total2 = float(np.sum(err2p))
    costs = [P.pivbos_plan_bins(err2n, err2p, steps, cnt, 3, f * total2, SEGMENTS)[2]["cost"]
             for f in (0.0, 0.01, 0.03, 0.1, 0.3, 1.0, 3.0)]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(costs, costs[1:])), costs


def test_limits_of_the_budget(P):
    err2n, err2p, steps, cnt = _bins(7)
    err2p[:20] = 0.0                             # bins the projection predicts exactly
    err2n[:20] = 0.0
    elig = cnt >= 3
    # no budget: only bins predicted without error can be served, and are
    # exactly when the projection costs less than the fallback
    served, network, m = P.pivbos_plan_bins(err2n, err2p, steps, cnt, 3, 0.0, SEGMENTS)
    exact = (err2p == 0.0) & elig & (cnt > 0)
    cheaper = PROJ * cnt < steps + FB_FIXED * cnt
    assert m["err2"] == 0.0
    assert np.array_equal(served, exact & cheaper)
    assert not np.any(network)                   # the correction costs more and gains nothing here
    # unlimited budget: every eligible bin whose projection is cheaper than
    # its fallback is served by the projection alone, no other
    served, network, m = P.pivbos_plan_bins(err2n, err2p, steps, cnt, 3, 1e300, SEGMENTS)
    assert np.array_equal(served, elig & (cnt > 0) & cheaper)
    assert not np.any(network)


def test_network_serves_where_the_projection_alone_cannot(P):
    """Two kinds of bins of equal size and steps: the projection's error is
    large on half of them and the network's correction removes most of it.
    With a budget below the projection's total error but above the
    corrected one, the plan serves every bin, correcting the bad ones."""
    n = 64
    cnt = np.full(n, 40)
    steps = np.full(n, 40 * 80.0)
    err2p = np.where(np.arange(n) % 2 == 0, 1e-6, 1e-3) * cnt
    err2n = np.where(np.arange(n) % 2 == 0, 1e-6, 1e-6) * cnt
    budget2 = 0.5 * float(np.sum(err2p))
    served, network, m = P.pivbos_plan_bins(err2n, err2p, steps, cnt, 1, budget2, SEGMENTS)
    assert np.all(served)
    assert np.array_equal(network, np.arange(n) % 2 == 1)
    served_p, network_p, m_p = P.pivbos_plan_bins(err2n, err2p, steps, cnt, 1, budget2, SEGMENTS, with_net=False)
    assert not np.any(network_p) and m_p["rays"] < m["rays"] and m_p["cost"] > m["cost"]


def test_rejects_bad_arguments(P):
    T = P.testing_lib()
    z = np.zeros(32)
    c = np.zeros(32, dtype=np.uint32)
    w = np.zeros(1, dtype=np.uint32)
    out = np.zeros(5)
    args = [z.ctypes.data, z.ctypes.data, z.ctypes.data, c.ctypes.data]
    assert T.pivbos_plan_bins(*args, 31, 1, 1.0, 1, 1, w.ctypes.data, w.ctypes.data, out.ctypes.data) == \
        P.ERR_INVALID_ARG
    assert T.pivbos_plan_bins(*args, 32, 1, -1.0, 1, 1, w.ctypes.data, w.ctypes.data, out.ctypes.data) == \
        P.ERR_INVALID_ARG
    assert T.pivbos_plan_bins(None, *args[1:], 32, 1, 1.0, 1, 1, w.ctypes.data, w.ctypes.data, out.ctypes.data) == \
        P.ERR_INVALID_ARG
