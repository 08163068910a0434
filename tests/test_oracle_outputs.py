"""Pins of the oracle's measured outputs against hand-computed values of Eq. 8-9,
exact constant-speed integrals, brute-force reconstruction from the simulated state
(traversal times, Sec. 6.3.1; per-edge samples, Sec. 6.4), an independent SplitMix64
from its published definition (reroute subsets), and the invariants of the decaying
reroute (Sec. 6.3.1)."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import dijkstra

import oracle as O
from paper_1807_01148_gb300 import scenarios as S

from .nets import make_net, scenario

MPH = 0.44704   # m/s per mile per hour (exact)


# ---------------------------------------------------------------- Eq. 8 (CO)
def test_co_rate_hand_values():
    # Eq. 8 at 0 mph: -0.064 + 0.00026 * 50^2 = 0.586 g/s; at 50 mph: -0.064 + 0.28 = 0.216
    assert math.isclose(O.oracle_co_rate(0.0), 0.586, rel_tol=1e-6)
    assert math.isclose(O.oracle_co_rate(50 * MPH), 0.216, rel_tol=1e-5)
    # 60 mph: -0.064 + 0.336 + 0.026 = 0.298
    assert math.isclose(O.oracle_co_rate(60 * MPH), 0.298, rel_tol=1e-5)


def test_co_rate_minimum_in_mph():
    # the parabola's vertex sits at 50 - 0.0056 / (2 * 0.00026) = 39.2308 mph, where the
    # rate is 0.18585 g/s; with the speed wrongly taken in m/s the vertex would be elsewhere
    vm = np.linspace(30.0, 48.0, 1801)
    rates = np.array([O.oracle_co_rate(np.float32(x * MPH)) for x in vm])
    assert abs(vm[rates.argmin()] - 39.2308) < 0.02
    assert math.isclose(rates.min(), 0.185846, rel_tol=1e-4)


# ---------------------------------------------------------------- Eq. 9 (fuel)
def test_fuel_rate_idle_and_cruise():
    assert math.isclose(O.oracle_fuel_rate(0.0, 0.0), 0.666, rel_tol=1e-7)
    assert math.isclose(O.oracle_fuel_rate(0.0, 1.5), 0.666, rel_tol=1e-7)      # v = 0: no power
    # 10 m/s cruise: 0.666 + 0.072 * (2.69 + 1.71 + 0.672) = 1.031184 mL/s
    assert math.isclose(O.oracle_fuel_rate(10.0, 0.0), 1.031184, rel_tol=1e-6)
    # 20 m/s, a = -0.1: 0.666 + 0.072 * (5.38 + 6.84 + 5.376 - 3.36) = 1.690992
    assert math.isclose(O.oracle_fuel_rate(20.0, -0.1), 1.690992, rel_tol=1e-6)


def test_fuel_rate_engine_drag_only_when_accelerating():
    # 10 m/s, a = 1: bracket 5.072 + 16.8 + P_ea (0.79296 * 1 * 10 = 7.9296) -> 2.8117152
    assert math.isclose(O.oracle_fuel_rate(10.0, 1.0), 2.8117152, rel_tol=1e-6)
    # the inertia term is odd in a and P_ea appears for a > 0 only
    for v, a in ((20.0, 0.1), (15.0, 0.05), (25.0, 0.2)):   # -a stays above the idle floor
        d = O.oracle_fuel_rate(v, a) - O.oracle_fuel_rate(v, -a)
        assert math.isclose(d, 0.072 * (2 * 1.680 * a * v + 0.79296 * a * a * v), rel_tol=1e-4)


def test_fuel_rate_idles_under_hard_braking():
    # negative tractive power: the engine idles at 0.666 mL/s, the rate never goes below
    assert O.oracle_fuel_rate(10.0, -2.0) == np.float32(0.666)
    assert O.oracle_fuel_rate(30.0, -4.0) == np.float32(0.666)
    vs = np.linspace(0, 35, 36)
    for a in (-3.0, -1.0, 0.0, 1.0):
        assert min(O.oracle_fuel_rate(float(v), a) for v in vs) >= np.float32(0.666)


# ---------------------------------------------------------------- integration along a run
def _one_link(length=5000.0, speed=20.0, lanes=1):
    return make_net([(0, 0), (length, 0)], [(0, 1)], lanes=lanes, length=length, speed=speed)


def test_emissions_constant_speed_closed_form():
    # a lone vehicle at its desired speed has a = 0 exactly: n steps burn n * dt * f(v0, 0)
    # and emit n * dt * P(v0)
    v0 = 20.0
    sc = scenario(_one_link(speed=v0), [[0]], state=dict(x=[0.0], v=[v0]))
    o = O.OracleSim(sc)
    o.set_routes(sc["routes"]["offsets"], sc["routes"]["links"])
    o.set_outputs(1)
    o.write_state(sc["init_state"])
    n = 200
    o.step(n)
    fuel, co = o.emissions()
    assert o.state()["v"][0] == np.float32(v0)
    f = 0.666 + 0.072 * (0.269 * v0 + 0.0171 * v0 ** 2 + 0.000672 * v0 ** 3)
    vm = v0 / MPH
    p = -0.064 + 0.0056 * vm + 0.00026 * (vm - 50) ** 2
    assert math.isclose(fuel[0], n * 0.5 * f, rel_tol=2e-6)
    assert math.isclose(co[0], n * 0.5 * p, rel_tol=2e-6)


def test_emissions_use_start_of_step_speed():
    # from standstill the first step runs at v = 0: idle fuel and the 0-mph CO rate, times dt
    sc = scenario(_one_link(), [[0]], state=dict(x=[0.0], v=[0.0]))
    o = O.OracleSim(sc)
    o.set_routes(sc["routes"]["offsets"], sc["routes"]["links"])
    o.set_outputs(1)
    o.write_state(sc["init_state"])
    o.step(1)
    fuel, co = o.emissions()
    assert math.isclose(fuel[0], 0.666 * 0.5, rel_tol=1e-6)
    assert math.isclose(co[0], 0.586 * 0.5, rel_tol=1e-6)
    o.step(1)   # second step: v = a dt = 0.5 m/s, a just below 1: power-based rate above idle
    assert o.emissions()[0][0] > 2 * 0.666 * 0.5


def test_emissions_stop_growing_after_arrival_and_before_departure():
    sc = S.small_grid()
    o = O.OracleSim(sc)
    o.route()
    o.set_outputs(1)
    o.step(400)
    st = o.state()
    fuel, co = o.emissions()
    assert (fuel[st["status"] == S.ST_PENDING] == 0).all()
    # a trip inserted in step t starts moving in step t + 1
    moved = (st["status"] != S.ST_PENDING) & (st["insert_step"] < 399)
    assert moved.sum() > 50
    assert (fuel[moved] > 0).all() and (co[moved] > 0).all()
    assert (fuel[st["insert_step"] == 399] == 0).all()
    arrived = st["status"] == S.ST_ARRIVED
    assert arrived.any()
    o.step(100)
    f2, c2 = o.emissions()
    assert (f2[arrived] == fuel[arrived]).all() and (c2[arrived] == co[arrived]).all()
    # each active step burns at least the idle rate
    steps = np.where(arrived, st["arrive_step"] - st["insert_step"] + 1, 0)
    assert (f2[arrived] >= 0.666 * 0.5 * steps[arrived] * (1 - 1e-6)).all()


# ---------------------------------------------------------------- traversal times
def _trajectory_traversals(o, n_steps):
    """Traversal times rebuilt from one state read per step: a trip that is pending at t
    and active at t + 1 entered its first link at step t; a link change or an arrival
    between t and t + 1 is an exit at step t."""
    nl = o.n_links
    s = np.zeros(nl, np.int64)
    n = np.zeros(nl, np.int32)
    enter = {}
    prev = o.state()
    for t0 in range(n_steps):
        t = o.counters()["t"]
        o.step(1)
        cur = o.state()
        for i in range(o.n_trips):
            if prev["status"][i] == S.ST_PENDING and cur["status"][i] == S.ST_ACTIVE:
                enter[i] = t
            elif prev["status"][i] == S.ST_ACTIVE:
                e = prev["link"][i]
                left = cur["status"][i] == S.ST_ARRIVED or cur["cursor"][i] != prev["cursor"][i]
                if left and i in enter:
                    s[e] += t - enter[i]
                    n[e] += 1
                if left and cur["status"][i] == S.ST_ACTIVE:
                    enter[i] = t
        prev = cur
    return s, n


def test_traversal_times_match_trajectory():
    sc = S.small_grid()
    o = O.OracleSim(sc)
    o.route()
    o.set_outputs(2)
    bs, bn = _trajectory_traversals(o, 500)
    s, n = o.link_times()
    assert n.sum() > 100
    np.testing.assert_array_equal(n, bn)
    np.testing.assert_array_equal(s, bs)


def test_traversal_time_free_road_constant_speed():
    # a lone vehicle at 20 m/s moves 10 m per 0.5 s step: a 100 m link takes 10 steps
    net = make_net([(0, 0), (100, 0), (200, 0), (300, 0), (400, 0)], [(0, 1), (1, 2), (2, 3), (3, 4)],
                   lanes=1, length=100.0, speed=20.0)
    sc = scenario(net, [[0, 1, 2, 3]], state=dict(x=[0.0], v=[20.0]))
    o = O.OracleSim(sc)
    o.set_routes(sc["routes"]["offsets"], sc["routes"]["links"])
    o.set_outputs(2)
    o.write_state(sc["init_state"])
    o.step(60)
    s, n = o.link_times()
    # link 0 was entered before the run (unknown entry): not measured
    np.testing.assert_array_equal(n, [0, 1, 1, 1])
    np.testing.assert_array_equal(s, [0, 10, 10, 10])


def test_measured_costs_rounding_and_gap():
    sc = S.small_grid()
    o = O.OracleSim(sc)
    o.route()
    o.set_outputs(2)
    o.step(600)
    s, n = o.link_times()
    prev = np.array([O.oracle_link_cost(float(L), float(v), 1, 0) for L, v in
                     zip(sc["network"]["link_length_m"], sc["network"]["link_speed_mps"])], np.int32)
    cost, gap = o.measured_costs(prev)
    dt_ds = 5
    num = den = 0
    for e in range(len(n)):
        if n[e] == 0:
            assert cost[e] == prev[e]
            continue
        mean = Fraction(int(s[e]) * dt_ds, int(n[e]))
        want = max(1, min(10 ** 6, math.floor(mean + Fraction(1, 2))))
        assert cost[e] == want
        num += int(n[e]) * abs(want - int(prev[e]))
        den += int(n[e]) * int(prev[e])
    assert gap == pytest.approx(num / den, rel=1e-15)
    # measured traversals include queueing and acceleration: never below free flow on average
    used = n > 0
    assert (cost[used] >= prev[used] - 1).mean() > 0.95


# ---------------------------------------------------------------- per-edge samples (Sec. 6.4)
def test_edge_samples_match_brute_force():
    sc = S.small_grid()
    net, par = sc["network"], sc["params"]
    o = O.OracleSim(sc)
    o.route()
    every, per, maxw = 20, 3, 12
    o.set_outputs(4, every, per, maxw)
    nl = o.n_links
    lanes = net["link_lanes"].astype(np.float64)
    L = net["link_length_m"].astype(np.float32).astype(np.float64)
    s0 = np.float64(np.float32(par["s0"][0]))
    cap = (L * lanes) / (np.float64(np.float32(par["veh_len"])) + s0)
    vfree = net["link_speed_mps"].astype(np.float32).astype(np.float64)
    su = np.zeros((maxw, nl))
    ss = np.zeros((maxw, nl))
    cnt = np.zeros(maxw, int)
    T = every * per * 10
    for t in range(T):
        if t % every == 0:
            st = o.state()
            act = np.where(st["status"] == S.ST_ACTIVE)[0]
            w = (t // every) // per
            for e in range(nl):
                on = [i for i in act if st["link"][i] == e]
                on.sort(key=lambda i: (st["lane"][i], st["x"][i], i))
                tot = 0.0
                for i in on:
                    tot += float(st["v"][i])
                su[w, e] += len(on) / cap[e]
                ss[w, e] += tot / len(on) if on else vfree[e]
            cnt[w] += 1
        o.step(1)
    u, sp, ns = o.edge_samples()
    np.testing.assert_array_equal(ns, [per] * 10 + [0, 0])
    np.testing.assert_allclose(u[:10], su[:10] / per, rtol=1e-13, atol=0)
    np.testing.assert_allclose(sp[:10], ss[:10] / per, rtol=1e-13, atol=0)
    assert (u[10:] == 0).all()
    assert u.max() > 0.05


def test_edge_samples_empty_network_is_free_flow():
    sc = S.small_grid()
    sc["demand"]["depart_step"][:] = 10 ** 6
    o = O.OracleSim(sc)
    o.route()
    o.set_outputs(4, 120, 6, 2)
    o.step(720)
    u, sp, ns = o.edge_samples()
    assert ns[0] == 6 and ns[1] == 0
    assert (u[0] == 0).all()
    np.testing.assert_array_equal(sp[0], sc["network"]["link_speed_mps"].astype(np.float32).astype(np.float64))


def test_edge_samples_window_capacity_enforced():
    sc = S.small_grid()
    o = O.OracleSim(sc)
    o.route()
    o.set_outputs(4, 10, 2, 3)     # windows cover steps 0 .. 59
    o.step(60)
    with pytest.raises(O.oracle.OracleError):
        o.step(1)


# ---------------------------------------------------------------- reroute subsets (Sec. 6.3.1)
def _splitmix64(z):
    """SplitMix64 from Steele, Lea & Flood (2014): increment, then the finaliser."""
    m = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def test_splitmix64_reference_first_output():
    # published first output of the generator seeded with 0
    assert _splitmix64(0) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("seed", [0, 1807011480, 2 ** 64 - 1])
def test_reroute_selection_is_splitmix_top16(seed):
    for vid in (0, 1, 77, 12345, 2 ** 31 - 1):
        for rnd in (1, 2, 3):
            top = _splitmix64(seed ^ ((vid << 32) | 0x80000000 | rnd)) >> 48
            for frac in (0, 1, 16384, 32768, 65535, 65536):
                assert O.oracle_reroute_selected(seed, vid, rnd, frac) == (top < frac)


def test_reroute_selection_fraction():
    n = 20000
    for frac, p in ((65536, 1.0), (32768, 0.5), (16384, 0.25), (0, 0.0)):
        got = np.mean([O.oracle_reroute_selected(S.BASE_SEED, i, 3, frac) for i in range(n)])
        assert abs(got - p) < 4 * math.sqrt(p * (1 - p) / n) + 1e-12


def _sp_cost(sc, cost, o_node, d_node):
    net = sc["network"]
    g = csr_matrix((cost.astype(float), (net["link_from"], net["link_to"])), shape=(net["n_nodes"],) * 2)
    # parallel links: csr_matrix sums duplicates, so keep the minimum by hand
    best = {}
    for e, (a, b) in enumerate(zip(net["link_from"], net["link_to"])):
        best[(a, b)] = min(best.get((a, b), 1e18), cost[e])
    rows, cols = zip(*best.keys())
    g = csr_matrix((list(best.values()), (rows, cols)), shape=(net["n_nodes"],) * 2)
    return dijkstra(g, indices=o_node)[d_node]


def test_reroute_keeps_unselected_and_shortest_for_selected():
    sc = S.small_grid()
    o = O.OracleSim(sc)
    o.route()
    off0, links0 = o.routes()
    rng = np.random.default_rng(3)
    cost = rng.integers(20, 400, o.n_links).astype(np.int32)
    o.reroute(cost, 32768, 2)
    off1, links1 = o.routes()
    ref = O.OracleSim(sc)
    ref.route(cost)
    off2, links2 = ref.routes()
    dem = sc["demand"]
    n_sel = 0
    for i in range(dem["n_trips"]):
        r0, r1, r2 = links0[off0[i]:off0[i + 1]], links1[off1[i]:off1[i + 1]], links2[off2[i]:off2[i + 1]]
        if O.oracle_reroute_selected(sc["params"]["seed"], i, 2, 32768):
            n_sel += 1
            np.testing.assert_array_equal(r1, r2)
            assert cost[r1].sum() == _sp_cost(sc, cost, dem["origin"][i], dem["dest"][i])
        else:
            np.testing.assert_array_equal(r1, r0)
    assert 0.4 < n_sel / dem["n_trips"] < 0.6
    assert o.counters()["t"] == 0


def test_reroute_all_equals_route_and_none_keeps():
    sc = S.small_grid()
    rng = np.random.default_rng(5)
    cost = rng.integers(20, 400, sc["network"]["n_links"]).astype(np.int32)
    a, b = O.OracleSim(sc), O.OracleSim(sc)
    a.route()
    a.reroute(cost, 65536, 1)
    b.route(cost)
    for x, y in zip(a.routes(), b.routes()):
        np.testing.assert_array_equal(x, y)
    c = O.OracleSim(sc)
    c.route()
    before = c.routes()
    c.reroute(cost, 0, 1)
    for x, y in zip(before, c.routes()):
        np.testing.assert_array_equal(x, y)


# ---------------------------------------------------------------- decaying equilibrium
def _two_route(n_trips=240, spacing=2):
    # 0 -> 1 -> 3: 2 x 400 m single-lane links at 25 m/s (32 s free flow), stop sign at 1
    # 0 -> 2 -> 3: 2 x 600 m single-lane links at 25 m/s (48 s free flow), stop sign at 2
    xy = [(0, 0), (400, 0), (300, 520), (800, 0)]
    links = [(0, 1), (1, 3), (0, 2), (2, 3)]
    net = make_net(xy, links, ctrl=[0, S.CTRL_STOP, S.CTRL_STOP, 0], lanes=1,
                   length=[400.0, 400.0, 600.0, 600.0], speed=25.0)
    sc = scenario(net, [[0, 1]] * n_trips, depart=np.arange(n_trips) * spacing)
    sc["params"]["cost_mode"] = 0
    return sc


def test_equilibrium_first_iteration_all_on_free_flow_path():
    sc = _two_route()
    o = O.OracleSim(sc)
    o.set_outputs(2)
    cost, gap = o.equilibrium([65536], 900)
    off, links = o.routes()
    assert (links.reshape(-1, 2) == [0, 1]).all()
    assert gap[0] > 0.05         # congestion made the fast path slower than its free-flow cost
    assert cost[0] > 160         # 0 -> 1 measured above its 16 s free-flow time


def test_equilibrium_loop_is_reroute_with_previous_measurement():
    sc = _two_route()
    fr = [65536, 65536, 32768, 16384]
    a = O.OracleSim(sc)
    a.set_outputs(2)
    cost_a, gap_a = a.equilibrium(fr, 900)
    b = O.OracleSim(sc)
    b.set_outputs(2)
    cost = np.array([O.oracle_link_cost(float(L), float(v), int(k), 0) for L, v, k in
                     zip(sc["network"]["link_length_m"], sc["network"]["link_speed_mps"],
                         sc["network"]["link_lanes"])], np.int32)
    gaps = []
    for k in range(4):
        if k == 0:
            b.route(cost)
        else:
            before = b.routes()
            b.reroute(cost, fr[k], k)
            off, links = b.routes()
            for i in range(b.n_trips):
                r = links[off[i]:off[i + 1]]
                if O.oracle_reroute_selected(sc["params"]["seed"], i, k, fr[k]):
                    assert cost[r].sum() == _sp_cost(sc, cost, 0, 3)
                else:
                    np.testing.assert_array_equal(r, before[1][before[0][i]:before[0][i + 1]])
        b.step(900)
        cost, g = b.measured_costs(cost)
        gaps.append(g)
    np.testing.assert_array_equal(cost, cost_a)
    np.testing.assert_array_equal(gaps, gap_a)
    # the adaptation spreads the demand over both paths and closes the gap
    off, links = b.routes()
    first = links[off[:-1]]
    assert 0 < (first == 0).sum() < b.n_trips
    assert gaps[1] < gaps[0] and gaps[3] <= gaps[1]


def test_mid_run_clear_restarts_windows():
    # cleared at t = 130 with samples every 60 steps, windows of 2: the next instant is 180
    # (sample 3), so window 1 closes with that one sample and window 2 with two
    sc = S.small_grid()
    o = O.OracleSim(sc)
    o.route()
    o.set_outputs(7, 60, 2, 16)
    o.step(130)
    assert o.edge_samples()[2][0] == 2
    o.reset_outputs()
    assert (o.emissions()[0] == 0).all() and (o.link_times()[1] == 0).all()
    assert (o.edge_samples()[2] == 0).all()
    st = o.state()
    o.step(500)
    n = o.edge_samples()[2]
    assert n[0] == 0 and n[1] == 1 and (n[2:5] == 2).all()
    # trips on a link at the clear are not counted on that link
    s, cnt = o.link_times()
    first_exit = cnt.sum()
    assert first_exit > 0
    del st
