"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle, bit-exact.

Routes (integer link ids), per-lane occupancy (lane_start and sorted trip ids), lane
decisions, counters and every binary32 state bit must be identical at every checked
step.  Cases span several lanes per link, signals, stop signs, ragged lane segments,
departures and arrivals."""
import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

from .parity import compare, run_lockstep, setup_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1807_01148_gb300 import gbtraffic
    return gbtraffic


@pytest.fixture(scope="module")
def O():
    import oracle
    return oracle


def test_routes_grid20(G, O):
    sc = S.grid()
    g, o = setup_pair(sc, G.Sim, O.OracleSim)
    og, lg = g.routes()
    oo, lo = o.routes()
    assert np.array_equal(og, oo)
    assert np.array_equal(lg, lo)


def test_routes_small_metro(G, O):
    sc = S.small_metro()
    g, o = setup_pair(sc, G.Sim, O.OracleSim)
    og, lg = g.routes()
    oo, lo = o.routes()
    assert np.array_equal(og, oo)
    assert np.array_equal(lg, lo)


def test_ring_bitexact(G, O):
    sc = S.ring()
    g, o = setup_pair(sc, G.Sim, O.OracleSim)
    run_lockstep(g, o, 3600, 400)


def test_small_grid_bitexact(G, O):
    sc = S.small_grid()
    g, o = setup_pair(sc, G.Sim, O.OracleSim)
    run_lockstep(g, o, 900, 30)


def test_small_metro_bitexact(G, O):
    sc = S.small_metro()
    g, o = setup_pair(sc, G.Sim, O.OracleSim)
    run_lockstep(g, o, 1200, 40)
