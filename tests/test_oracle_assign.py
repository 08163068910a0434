"""Pins of the oracle's static user equilibrium (Sec. 5.2, Eq. 6) with BPR link times
(Eq. 3): closed forms on one link, the Wardrop point of two parallel links solved
independently (scipy brentq), an independent path-flow optimiser (scipy SLSQP over all
simple paths) on a Braess-type network, all-or-nothing flows against the routes of
orc_route, flow conservation at every node, and the descent of the objective."""
import math

import networkx as nx
import numpy as np
import pytest
from scipy.optimize import brentq, minimize

import oracle as O
from paper_1807_01148_gb300 import scenarios as S

from .nets import make_net


def _od_scenario(net, od_pairs):
    """Trips given as (origin node, destination node) pairs; routes are planned later."""
    o = np.array([a for a, _ in od_pairs], np.int32)
    d = np.array([b for _, b in od_pairs], np.int32)
    return dict(name="assign", network=net, demand=S._demand(o, d, np.zeros(len(o), np.int32)),
                params=S.default_params(1))


def test_bpr_single_link_closed_form():
    # one 1000 m link at 10 m/s (t0 = 100 s, Eq. 4), capacity 1000, 2000 trips
    net = make_net([(0, 0), (1000, 0)], [(0, 1)], lanes=1, length=1000.0, speed=10.0)
    o = O.OracleSim(_od_scenario(net, [(0, 1)] * 2000))
    r = o.assign_static([1000.0], alpha=0.15, beta=4, max_iter=3)
    assert r["flow"][0] == 2000.0
    assert math.isclose(r["time"][0], 100.0 * (1 + 0.15 * 2 ** 4), rel_tol=1e-14)      # 340 s
    # Beckmann term: int_0^x t0 (1 + a (s/c)^4) ds = t0 x (1 + a (x/c)^4 / 5) = 296000
    assert math.isclose(r["objective"][0], 296000.0, rel_tol=1e-12)
    r1 = o.assign_static([1000.0], alpha=0.15, beta=1, max_iter=1)
    assert math.isclose(r1["time"][0], 130.0, rel_tol=1e-14)
    np.testing.assert_array_equal(r["gap"], 0.0)                   # one path: nothing to shift


@pytest.mark.parametrize("t0b,D", [(150.0, 3000), (120.0, 1500), (400.0, 5000)])
def test_two_parallel_links_wardrop(t0b, D):
    # parallel links 0 -> 1, free-flow 100 s and t0b s, capacity 1000 each: the exact line
    # search of the first iteration lands on the point where both times are equal
    L = [1000.0, t0b * 10.0]
    net = make_net([(0, 0), (1000, 0)], [(0, 1), (0, 1)], lanes=1, length=L, speed=10.0)
    o = O.OracleSim(_od_scenario(net, [(0, 1)] * D))
    r = o.assign_static([1000.0, 1000.0], alpha=0.15, beta=4, max_iter=2, bisect_iter=40)

    def tt(t0, x):
        return t0 * (1 + 0.15 * (x / 1000.0) ** 4)
    if tt(100.0, D) <= t0b:
        xa = float(D)            # the slow link stays unused
    else:
        xa = brentq(lambda x: tt(100.0, x) - tt(t0b, D - x), 0.0, D, xtol=1e-12)
    assert abs(r["flow"][0] - xa) < 1e-6 * D
    assert abs(r["flow"].sum() - D) < 1e-9 * D
    if xa < D:
        assert math.isclose(r["time"][0], r["time"][1], rel_tol=1e-6)
        assert 0.0 < r["step"][0] < 1.0


def _braess():
    # s=0, a=1, b=2, t=3; 0->1 and 2->3 congestible, 1->3 and 0->2 long and wide, 1->2 a
    # short bridge; a second OD pair 1 -> 3 shares the network
    xy = [(0, 0), (1000, 600), (1000, -600), (2000, 0)]
    links = [(0, 1), (1, 3), (0, 2), (2, 3), (1, 2)]
    length = [800.0, 2500.0, 2500.0, 800.0, 200.0]
    lanes = [1, 3, 3, 1, 1]
    net = make_net(xy, links, lanes=lanes, length=length, speed=20.0)
    cap = np.array([400.0, 3000.0, 3000.0, 400.0, 1000.0])
    trips = [(0, 3)] * 900 + [(1, 3)] * 250
    return net, cap, trips


def _beckmann(t0, cap, x, a=0.15, b=4):
    return float(np.sum(t0 * x * (1 + a * (x / cap) ** b / (b + 1))))


def test_matches_independent_path_flow_optimum():
    net, cap, trips = _braess()
    o = O.OracleSim(_od_scenario(net, trips))
    r = o.assign_static(cap, max_iter=300, bisect_iter=40)
    t0 = net["link_length_m"].astype(np.float64) / net["link_speed_mps"].astype(np.float64)
    # independent optimum: Beckmann objective over the flows of every simple path
    G = nx.MultiDiGraph()
    for e, (u, v) in enumerate(zip(net["link_from"], net["link_to"])):
        G.add_edge(int(u), int(v), key=e)
    demand = {}
    for od in trips:
        demand[od] = demand.get(od, 0) + 1
    cols, rows = [], []
    for od, dem in demand.items():
        paths = [[e for (_, _, e) in p] for p in nx.all_simple_edge_paths(G, od[0], od[1])]
        rows.append((len(cols), len(cols) + len(paths), dem))
        cols += paths
    A = np.zeros((len(t0), len(cols)))
    for j, p in enumerate(cols):
        A[p, j] = 1.0

    def f(h):
        return _beckmann(t0, cap, A @ h)
    cons = [{"type": "eq", "fun": (lambda h, a=a, b=b, d=d: h[a:b].sum() - d)} for a, b, d in rows]
    h0 = np.concatenate([np.full(b - a, d / (b - a)) for a, b, d in rows])
    best = minimize(f, h0, method="SLSQP", bounds=[(0, None)] * len(cols), constraints=cons,
                    options={"ftol": 1e-14, "maxiter": 2000})
    assert best.success
    fstar = best.fun
    fw = r["objective"][-1]
    assert math.isclose(fw, _beckmann(t0, cap, r["flow"]), rel_tol=1e-12)
    # f(x_K) is feasible, hence >= f*; and within the last duality gap of it
    tx = float(np.sum(r["time"] * r["flow"]))
    assert fw >= fstar * (1 - 1e-9)
    assert fw - fstar <= max(r["gap"][-1], 0.0) * tx + 1e-6 * fstar
    np.testing.assert_allclose(r["flow"], A @ best.x, rtol=2e-2, atol=2.0)
    # Wardrop: the bridge is used and the used paths of the main pair have equal times
    used = [p for p, hj in zip(cols, best.x) if hj > 1.0 and p[0] in (0, 2)]
    times = [r["time"][p].sum() for p in used]
    assert max(times) - min(times) < 1e-2 * max(times)


def test_aon_equals_counts_of_planned_routes():
    sc = S.small_grid()
    o = O.OracleSim(sc)
    cost = np.array([O.oracle_link_cost(float(L), float(v), 1, 0) for L, v in
                     zip(sc["network"]["link_length_m"], sc["network"]["link_speed_mps"])], np.int32)
    flow = o.aon(cost)
    o.route(cost)
    off, links = o.routes()
    np.testing.assert_array_equal(flow, np.bincount(links, minlength=o.n_links).astype(np.float64))


def test_flow_conservation_and_descent_small_grid():
    sc = S.small_grid(n_trips=1500)
    cap = S.bpr_capacity(sc, 0.05)     # congested: volume / capacity of order 1 on busy links
    o = O.OracleSim(sc)
    r = o.assign_static(cap, max_iter=25)
    net, dem = sc["network"], sc["demand"]
    nn = net["n_nodes"]
    out_f = np.bincount(net["link_from"], weights=r["flow"], minlength=nn)
    in_f = np.bincount(net["link_to"], weights=r["flow"], minlength=nn)
    net_dem = (np.bincount(dem["dest"], minlength=nn) - np.bincount(dem["origin"], minlength=nn)).astype(float)
    np.testing.assert_allclose(in_f - out_f, net_dem, atol=1e-6)
    obj = r["objective"]
    assert (np.diff(obj) <= 1e-9 * obj[0]).all()            # exact line search: no ascent
    assert ((r["step"] >= 0) & (r["step"] <= 1)).all()
    assert r["gap"][-1] < 0.5 * r["gap"][0]
    assert (r["gap"] > -1e-3).all()
    t0 = net["link_length_m"].astype(np.float64) / net["link_speed_mps"].astype(np.float64)
    np.testing.assert_allclose(r["time"], t0 * (1 + 0.15 * (r["flow"] / cap) ** 4), rtol=1e-12)


def test_invalid_inputs():
    sc = S.small_grid()
    o = O.OracleSim(sc)
    cap = S.bpr_capacity(sc, 1.0)
    bad = cap.copy()
    bad[3] = 0.0
    for kw in (dict(capacity=bad), dict(capacity=cap, beta=0), dict(capacity=cap, beta=9),
               dict(capacity=cap, alpha=-1.0), dict(capacity=cap, max_iter=-1)):
        with pytest.raises(O.oracle.OracleError):
            o.assign_static(**kw)
