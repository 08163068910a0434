"""GPU parity of the static user equilibrium (Frank-Wolfe on BPR times, Sec. 5.2, Eq. 3,
Eq. 6) through the C ABI: flows, times, gaps, steps and objectives equal to the oracle's
in every bit on small networks, on the small metro, and on the full-size metro network
(550,000 links) with the trips of sampled origins; flow conservation of the full-demand
all-or-nothing assignment (3,000,000 trips, 225,000 trees); error codes."""
import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

from .nets import make_net

pytestmark = pytest.mark.gpu

KEYS = ("flow", "time", "gap", "step", "objective")


@pytest.fixture(scope="module")
def G():
    from paper_1807_01148_gb300 import gbtraffic
    return gbtraffic


@pytest.fixture(scope="module")
def O():
    import oracle
    return oracle


def _same(a, b, label):
    for k in KEYS:
        x, y = np.ascontiguousarray(a[k]), np.ascontiguousarray(b[k])
        bad = np.flatnonzero(x.view(np.uint64) != y.view(np.uint64))
        assert not len(bad), f"{label}: {k} differs at {bad[:8]}: {x[bad[:4]]} vs {y[bad[:4]]}"


def _both(G, O, sc, cap, **kw):
    g = G.Sim(sc)
    o = O.OracleSim(sc)
    return g.assign_static(cap, **kw), o.assign_static(cap, **kw)


@pytest.mark.parametrize("period_h,iters", [(0.05, 25), (0.02, 40), (1.0, 5)])
def test_assign_small_grid_bitexact(G, O, period_h, iters):
    sc = S.small_grid(n_trips=1500)
    a, b = _both(G, O, sc, S.bpr_capacity(sc, period_h), max_iter=iters)
    _same(a, b, f"grid period {period_h}")


def test_assign_braess_and_parallel_links_bitexact(G, O):
    xy = [(0, 0), (1000, 600), (1000, -600), (2000, 0)]
    links = [(0, 1), (1, 3), (0, 2), (2, 3), (1, 2), (0, 1)]
    net = make_net(xy, links, lanes=[1, 3, 3, 1, 1, 2], length=[800.0, 2500.0, 2500.0, 800.0, 200.0, 1400.0],
                   speed=20.0)
    od = [(0, 3)] * 900 + [(1, 3)] * 250 + [(0, 2)] * 120
    o_ = np.array([a for a, _ in od], np.int32)
    d_ = np.array([b for _, b in od], np.int32)
    sc = dict(name="braess", network=net, demand=S._demand(o_, d_, np.zeros(len(od), np.int32)),
              params=S.default_params(1))
    cap = np.array([400.0, 3000.0, 3000.0, 400.0, 1000.0, 600.0])
    for beta in (1, 4, 6):
        a, b = _both(G, O, sc, cap, beta=beta, max_iter=60, bisect_iter=40)
        _same(a, b, f"braess beta {beta}")


def test_assign_small_metro_bitexact(G, O):
    sc = S.small_metro(n_trips=20000)
    cap = S.bpr_capacity(sc, 0.5, S.METRO_EDGE_TYPES)
    a, b = _both(G, O, sc, cap, max_iter=12)
    _same(a, b, "small metro")
    assert a["gap"][-1] < a["gap"][0]


def test_assign_full_metro_network_sampled_origins(G, O):
    sc = S.metro()
    dem = sc["demand"]
    rng = np.random.default_rng(23)
    origins = rng.choice(np.unique(dem["origin"]), 40, replace=False)
    keep = np.flatnonzero(np.isin(dem["origin"], origins))
    sub = dict(sc, demand=S._demand(dem["origin"][keep], dem["dest"][keep], dem["depart_step"][keep]))
    cap = S.bpr_capacity(sc, 0.02, S.METRO_EDGE_TYPES)
    a, b = _both(G, O, sub, cap, max_iter=3)
    _same(a, b, "metro sampled origins")


def test_assign_full_metro_demand_conservation(G):
    sc = S.metro()
    net, dem = sc["network"], sc["demand"]
    g = G.Sim(sc)
    r = g.assign_static(S.bpr_capacity(sc, 24.0, S.METRO_EDGE_TYPES), max_iter=1)
    nn = net["n_nodes"]
    out_f = np.bincount(net["link_from"], weights=r["flow"], minlength=nn)
    in_f = np.bincount(net["link_to"], weights=r["flow"], minlength=nn)
    want = (np.bincount(dem["dest"], minlength=nn) - np.bincount(dem["origin"], minlength=nn)).astype(float)
    np.testing.assert_allclose(in_f - out_f, want, atol=1e-6 * dem["n_trips"])
    assert r["objective"][1] <= r["objective"][0]
    assert 0.0 <= r["step"][0] <= 1.0


def test_assign_error_codes(G):
    sc = S.small_grid()
    g = G.Sim(sc)
    cap = S.bpr_capacity(sc, 1.0)
    for kw in (dict(beta=0), dict(beta=9), dict(alpha=-0.1), dict(max_iter=-1), dict(bisect_iter=61)):
        with pytest.raises(G.SimError) as e:
            g.assign_static(cap, **kw)
        assert e.value.code == G.SIM_EINVAL
    bad = cap.copy()
    bad[0] = np.nan
    with pytest.raises(G.SimError) as e:
        g.assign_static(bad)
    assert e.value.code == G.SIM_EINVAL
    r = g.assign_static(cap, max_iter=0)       # the initial all-or-nothing assignment only
    assert len(r["objective"]) == 1 and r["flow"].sum() > 0
