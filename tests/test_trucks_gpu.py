"""GPU parity of vehicle types (Sec. 6.3.5 trucks: own length, acceleration scale and
maximum speed) through the C ABI: every bit of the state equal to the oracle's on the
small grid (with the measured outputs on as well), the 20x20 grid, a batched handle,
persistent execution and two full-size metro steps (3,000,000 vehicles); one car type
equal to the plain model; error codes."""
import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

from .parity import compare, diff_state, run_lockstep, setup_pair

pytestmark = pytest.mark.gpu

CAR = (5.0, 1.0, 1e9)
TRUCK = (12.0, 0.6, 24.0)
SEMI = (18.0, 0.45, 22.0)


@pytest.fixture(scope="module")
def G():
    from paper_1807_01148_gb300 import gbtraffic
    return gbtraffic


@pytest.fixture(scope="module")
def O():
    import oracle
    return oracle


def _mix(n, seed=7, shares=(0.75, 0.17, 0.08)):
    rng = np.random.default_rng(seed)
    return rng.choice(len(shares), size=n, p=shares).astype(np.uint8)


def _typed_pair(G, O, sc, types, tt):
    g, o = setup_pair(sc, G.Sim, O.OracleSim)
    g.set_vehicle_types(types, tt)
    o.set_vehicle_types(types, tt)
    return g, o


def test_trucks_small_grid_bitexact(G, O):
    sc = S.small_grid(n_trips=900)
    g, o = _typed_pair(G, O, sc, [CAR, TRUCK, SEMI], _mix(900))
    run_lockstep(g, o, 1200, 150)


def test_trucks_with_outputs_bitexact(G, O):
    sc = S.small_grid(n_trips=900, seed=S.BASE_SEED + 31)
    g, o = _typed_pair(G, O, sc, [CAR, TRUCK], _mix(900, shares=(0.7, 0.3)))
    g.set_outputs(7, 60, 3, 8)
    o.set_outputs(7, 60, 3, 8)
    g.step(900)
    o.step(900)
    compare(g, o, "trucks + outputs")
    for a, b in zip(g.emissions() + g.link_times() + g.edge_samples(), o.emissions() + o.link_times() + o.edge_samples()):
        assert np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


def test_trucks_grid20_bitexact(G, O):
    sc = S.grid()
    g, o = _typed_pair(G, O, sc, [CAR, TRUCK], _mix(sc["demand"]["n_trips"], shares=(0.85, 0.15)))
    run_lockstep(g, o, 3000, 1000)


def test_single_car_type_equals_plain(G):
    sc = S.small_grid()
    a = G.setup(sc)
    b = G.setup(sc)
    b.set_vehicle_types([(5.0, 1.0, 1e9)], np.zeros(sc["demand"]["n_trips"], np.uint8))
    a.step(800)
    b.step(800)
    assert not diff_state(a.state(), b.state())


def test_trucks_persistent_and_batched(G, O):
    scs = [S.small_grid(n=n, n_trips=150 * n, steps=700, seed=1300 + k, window_steps=400) for k, n in enumerate((5, 7))]
    tts = [_mix(sc["demand"]["n_trips"], seed=40 + k) for k, sc in enumerate(scs)]
    p = G.setup(scs[0])
    p.set_vehicle_types([CAR, TRUCK, SEMI], tts[0])
    p.set_exec(G.SIM_EXEC_PERSISTENT, threads=256, blocks_per_sm=1)
    o = O.OracleSim(scs[0])
    o.route()
    o.set_vehicle_types([CAR, TRUCK, SEMI], tts[0])
    p.step(600)
    o.step(600)
    compare(p, o, "persistent trucks")
    b = G.Sim.batch(scs)
    b.route()
    b.set_vehicle_types([CAR, TRUCK, SEMI], np.concatenate(tts))
    b.step(600)
    sb = b.state()
    base = link_base = 0
    for sc, tt in zip(scs, tts):
        o = O.OracleSim(sc)
        o.route()
        o.set_vehicle_types([CAR, TRUCK, SEMI], tt)
        o.step(600)
        n = sc["demand"]["n_trips"]
        sl = {k: v[base:base + n].copy() for k, v in sb.items()}
        act = sl["status"] == 1
        sl["link"][act] -= link_base
        assert not diff_state(sl, o.state())
        base += n
        link_base += sc["network"]["n_links"]


def test_trucks_metro_full_size_two_steps(G, O):
    sc = S.metro()
    off, links = S.random_walk_routes(sc, min_hops=10, max_hops=40)
    sc["routes"] = dict(offsets=off, links=links)
    sc["init_state"] = S.saturate(sc, off, links)
    tt = _mix(sc["demand"]["n_trips"], shares=(0.9, 0.07, 0.03))
    g, o = _typed_pair(G, O, sc, [CAR, TRUCK, SEMI], tt)
    for k in range(2):
        g.step(1)
        o.step(1)
        compare(g, o, f"metro trucks step {k + 1}", check_occ=(k == 1))


def test_vehicle_type_errors(G):
    sc = S.small_grid()
    g = G.setup(sc)
    n = sc["demand"]["n_trips"]
    with pytest.raises(G.SimError) as e:
        g.set_vehicle_types([CAR], np.ones(n, np.uint8))
    assert e.value.code == G.SIM_EINVAL
    with pytest.raises(G.SimError) as e:
        g.set_vehicle_types([(5.0, 0.0, 30.0)], np.zeros(n, np.uint8))
    assert e.value.code == G.SIM_EINVAL
    with pytest.raises(G.SimError) as e:
        g.set_vehicle_types([CAR] * 9, np.zeros(n, np.uint8))
    assert e.value.code == G.SIM_EINVAL
    g.set_vehicle_types([CAR, TRUCK], (np.arange(n) % 4 == 0).astype(np.uint8))
    with pytest.raises(G.SimError) as e:
        g.adjoint(20, 20, np.zeros((1, n)), 1)
    assert e.value.code == G.SIM_ESTATE
    g.set_vehicle_types([], None)
    g.write_state(g.state())
    g.adjoint(20, 20, np.zeros((1, n)), 1)
