"""Pins of the oracle's vehicle types (Sec. 6.3.5: trucks differ in size, acceleration
and maximum speed): one type equal to the single class is the plain model bit for bit;
a truck's first step from rest and its cruising speed (closed forms); a car behind a
truck settles at the IDM equilibrium gap behind the truck's rear; departures need s0 +
the entering vehicle's own length; the simultaneous-change rule measures with the longer
vehicle."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1807_01148_gb300 import scenarios as S

from .nets import make_net, scenario

CAR = (5.0, 1.0, 1e9)
TRUCK = (12.0, 0.5, 22.0)


def _run(sc, steps, types=None, trip_type=None):
    o = O.OracleSim(sc)
    if "routes" in sc:
        o.set_routes(sc["routes"]["offsets"], sc["routes"]["links"])
    else:
        o.route()
    if types is not None:
        o.set_vehicle_types(types, trip_type)
    if "init_state" in sc:
        o.write_state(sc["init_state"])
    o.step(steps)
    return o


def test_single_car_type_is_the_plain_model():
    sc = S.small_grid()
    a = _run(sc, 700)
    b = _run(sc, 700, [CAR], np.zeros(sc["demand"]["n_trips"], np.uint8))
    for k, v in a.state().items():
        assert np.array_equal(np.ascontiguousarray(v).view(np.uint8), np.ascontiguousarray(b.state()[k]).view(np.uint8)), k


def _road(length=20000.0, speed=30.0, lanes=1):
    return make_net([(0, 0), (length, 0)], [(0, 1)], lanes=lanes, length=length, speed=speed)


def test_truck_acceleration_and_speed_cap():
    sc = scenario(_road(), [[0]], state=dict(x=[0.0], v=[0.0]))
    o = _run(sc, 1, [CAR, TRUCK], [1])
    # first step from rest: a = 0.5 * 1.0 m/s^2 over dt = 0.5 s
    assert o.state()["v"][0] == np.float32(0.25)
    o.step(1500)
    # free road: the truck cruises at min(30, 22) m/s
    assert abs(o.state()["v"][0] - 22.0) < 1e-3
    c = _run(sc, 600, [CAR, TRUCK], [0])       # a car reaches the link's 30 m/s (before the road ends)
    assert c.state()["status"][0] == S.ST_ACTIVE
    assert abs(c.state()["v"][0] - 30.0) < 0.1


@pytest.mark.parametrize("lead_len", [5.0, 12.0, 18.0])
def test_car_behind_truck_keeps_equilibrium_gap_to_its_rear(lead_len):
    # leader: a vehicle capped at 15 m/s started at 15 m/s; follower: a car.  The car
    # settles at s_e(15) behind the leader's rear, s_e = (s0 + v T) / sqrt(1 - (v/v0)^4)
    vl = 15.0
    lead = (lead_len, 1.0, vl)
    sc = scenario(_road(80000.0), [[0], [0]], state=dict(x=[0.0, 60.0], v=[0.0, vl]))
    o = _run(sc, 4000, [CAR, lead], [0, 1])
    st = o.state()
    se = (2.0 + vl * 1.5) / math.sqrt(1 - (vl / 30.0) ** 4)
    gap = float(st["x"][1] - st["x"][0]) - lead_len
    assert abs(gap - se) < 2e-2, (gap, se)
    assert abs(float(st["v"][0]) - vl) < 1e-3


def test_departure_needs_own_length():
    # a car at x = 14 m leaves 9 m of rear space: a car (needs s0 + 5 = 7) enters at step
    # 0, a 12 m truck (needs 14) waits
    sc = scenario(_road(), [[0], [0]], state=dict(status=[1, 0], x=[14.0, 0.0], v=[0.0, 0.0]))
    car = _run(sc, 1, [CAR, TRUCK], [0, 0])
    assert car.state()["status"][1] == S.ST_ACTIVE and car.state()["insert_step"][1] == 0
    truck = _run(sc, 1, [CAR, TRUCK], [0, 1])
    assert truck.state()["status"][1] == S.ST_PENDING


def _corridor(lanes=3):
    return make_net([(0.0, 0.0), (1000.0, 0.0), (2000.0, 0.0)], [(0, 1), (1, 2)], lanes=lanes)


def test_conflicting_changes_measured_with_the_longer_vehicle():
    # A (vid 0, lane 0) and B (vid 1, lane 2), 10 m apart, close on vehicles standing near
    # the link end (too close to it to change lanes themselves) and move into free lane 1.
    # Cars: 10 m >= 5 + 2, both move.  A a 12 m truck: 10 m < 12 + 2, B is cancelled.
    net = _corridor()
    st = dict(lane=[0, 2, 0, 2], x=[960.0, 970.0, 995.0, 996.0], v=[20.0, 20.0, 0.0, 0.0])
    sc = scenario(net, [[0, 1]] * 4, st)
    long_truck = (12.0, 1.0, 1e9)
    cars = _run(sc, 1, [CAR, long_truck], [0, 0, 0, 0])
    assert cars.state()["lane_change"].tolist() == [1, -1, 0, 0]
    mixed = _run(sc, 1, [CAR, long_truck], [1, 0, 0, 0])
    assert mixed.state()["lane_change"].tolist() == [1, 0, 0, 0]


def test_invalid_types_and_adjoint_refused():
    sc = S.small_grid()
    o = O.OracleSim(sc)
    o.route()
    n = sc["demand"]["n_trips"]
    with pytest.raises(O.oracle.OracleError):
        o.set_vehicle_types([CAR], np.ones(n, np.uint8))        # type index out of range
    with pytest.raises(O.oracle.OracleError):
        o.set_vehicle_types([(0.0, 1.0, 30.0)], np.zeros(n, np.uint8))
    o.set_vehicle_types([CAR, TRUCK], (np.arange(n) % 5 == 0).astype(np.uint8))
    with pytest.raises(O.oracle.OracleError):
        o.adjoint(20, 20, np.zeros((1, n)), 1)
    o.set_vehicle_types([], None)
    o.adjoint(20, 20, np.zeros((1, n)), 1)
