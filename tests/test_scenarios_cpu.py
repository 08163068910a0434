"""The seeded workloads beyond the oracle pins (CPU): the jammed corridors hold the queues
they describe and discharge them through the signal under the oracle's model, and the
64-scenario ensemble has the sizes and parameter ranges it states."""
import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

PER_LANE = 2000 // 7          # vehicles per lane of a 2 km queue at 7 m spacing


def test_jammed_corridors_layout():
    sc = S.jammed_corridors(n_corr=3)
    net, st = sc["network"], sc["init_state"]
    assert (net["n_nodes"], net["n_links"]) == (9, 6)
    assert np.array_equal(net["link_length_m"], [2000.0, 200.0] * 3)
    assert np.array_equal(net["link_lanes"], [2] * 6)
    assert np.array_equal(net["node_control"], [S.CTRL_NONE, S.CTRL_SIGNAL, S.CTRL_NONE] * 3)
    n = sc["demand"]["n_trips"]
    assert n == 3 * 2 * PER_LANE
    assert (st["status"] == S.ST_ACTIVE).all() and not st["v"].any() and not st["cursor"].any()
    for c in range(3):
        on = st["link"] == 2 * c
        assert on.sum() == 2 * PER_LANE
        for lane in (0, 1):
            xs = np.sort(st["x"][on & (st["lane"] == lane)])
            assert len(xs) == PER_LANE
            assert xs[-1] == pytest.approx(1999.0)
            assert np.allclose(np.diff(xs), 7.0)           # 2 m gaps behind 5 m vehicles
    off, links = sc["routes"]["offsets"], sc["routes"]["links"]
    assert np.array_equal(np.diff(off), np.full(n, 2))
    first, second = links[off[:-1]], links[off[:-1] + 1]
    assert np.array_equal(first, st["link"]) and np.array_equal(second, st["link"] + 1)


def test_jammed_corridors_discharge_in_the_oracle():
    import oracle
    sc = S.jammed_corridors(n_corr=2)
    n = sc["demand"]["n_trips"]
    o = oracle.OracleSim(sc)
    o.set_routes(sc["routes"]["offsets"], sc["routes"]["links"])
    o.write_state(sc["init_state"])
    lane_start, _ = o.occupancy()
    assert np.diff(lane_start).max() == PER_LANE            # one lane segment per queue
    o.step(480)                                             # four signal cycles
    st, c = o.state(), o.counters()
    active, arrived = st["status"] == S.ST_ACTIVE, st["status"] == S.ST_ARRIVED
    assert active.sum() + arrived.sum() == n                 # nobody lost
    assert c["arrived"] == arrived.sum() and c["arrived"] > 0
    crossed = arrived | (active & (st["link"] % 2 == 1))
    # only green time lets vehicles through: about 15 s of every minute
    assert 0 < crossed.sum() < n // 4
    # the queue behind the line is still ordered, with positive gaps, in every lane
    long_link = active & (st["link"] % 2 == 0)
    for link in np.unique(st["link"][long_link]):
        for lane in (0, 1):
            xs = np.sort(st["x"][long_link & (st["link"] == link) & (st["lane"] == lane)])
            assert (np.diff(xs) > sc["params"]["veh_len"]).all()


def test_ensemble_sizes_and_parameters():
    scs = S.ensemble()
    assert len(scs) == 64 and all(sc["steps"] == 7200 for sc in scs)
    sides = []
    for sc in scs:
        side = int(round(sc["network"]["n_nodes"] ** 0.5))
        assert side * side == sc["network"]["n_nodes"] and side in (10, 15, 20, 30, 40)
        sides.append(side)
        assert sc["demand"]["n_trips"] == 5000 + 75000 * (side * side - 100) // 1500
        assert (sc["network"]["link_length_m"] == 200.0).all() and (sc["network"]["link_lanes"] == 2).all()
        p = sc["params"]
        assert 25 <= p["v0"][0] <= 33 and 1 <= p["T"][0] <= 2 and 0.8 <= p["a"][0] <= 1.5
        assert 1.2 <= p["b"][0] <= 2.5
        assert sc["demand"]["depart_step"].max() < 7200
    assert len(set(sides)) >= 4
    assert sum(sc["demand"]["n_trips"] for sc in scs) == 2_081_250
