"""GPU parity of the measured outputs and of the decaying equilibrium, through the C ABI:

- fuel and CO per trip (Eq. 8-9), link traversal sums (Sec. 6.3.1) and per-edge
  window means (Sec. 6.4): every bit equal to the oracle, on the small grid, the
  20x20 signalised grid and two full-size metro steps (3,000,000 vehicles), in graph
  and persistent execution, across a mid-run clear, and for a batched handle;
- the hash-selected reroute and the four-iteration equilibrium loop: identical routes,
  measured costs, gaps and states;
- the error codes of the new calls."""
import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

from .parity import compare, diff_state, setup_pair

pytestmark = pytest.mark.gpu

ALL = 7
SCHEDULE = [65536, 65536, 32768, 16384]


@pytest.fixture(scope="module")
def G():
    from paper_1807_01148_gb300 import gbtraffic
    return gbtraffic


@pytest.fixture(scope="module")
def O():
    import oracle
    return oracle


def _same_bits(a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def compare_outputs(g, o, flags, label=""):
    if flags & 1:
        fg, cg = g.emissions()
        fo, co = o.emissions()
        bad = np.flatnonzero(fg.view(np.uint64) != fo.view(np.uint64))
        assert not len(bad), f"{label}: fuel differs at trips {bad[:8]}: {fg[bad[:4]]} vs {fo[bad[:4]]}"
        assert _same_bits(cg, co), f"{label}: CO differs"
    if flags & 2:
        sg, ng = g.link_times()
        so, no = o.link_times()
        assert np.array_equal(ng, no), f"{label}: traversal counts differ at {np.flatnonzero(ng != no)[:8]}"
        assert np.array_equal(sg, so), f"{label}: traversal sums differ at {np.flatnonzero(sg != so)[:8]}"
    if flags & 4:
        ug, vg, kg = g.edge_samples()
        uo, vo, ko = o.edge_samples()
        assert np.array_equal(kg, ko), f"{label}: window sample counts {kg} vs {ko}"
        assert _same_bits(ug, uo), f"{label}: utilisation differs at {np.argwhere(ug != uo)[:8]}"
        assert _same_bits(vg, vo), f"{label}: speed differs at {np.argwhere(vg != vo)[:8]}"


def _pair(G, O, sc, flags=ALL, every=60, per=3, maxw=16):
    g, o = setup_pair(sc, G.Sim, O.OracleSim)
    g.set_outputs(flags, every, per, maxw)
    o.set_outputs(flags, every, per, maxw)
    return g, o


def test_outputs_small_grid_bitexact(G, O):
    g, o = _pair(G, O, S.small_grid())
    for k in range(8):
        g.step(300)
        o.step(300)
        compare(g, o, f"step {300 * (k + 1)}")
        compare_outputs(g, o, ALL, f"step {300 * (k + 1)}")
    u, _, n = g.edge_samples()
    assert (n[:13] == 3).all() and u.max() > 0
    assert g.link_times()[1].sum() > 1000 and g.emissions()[0].sum() > 0


def test_outputs_persistent_equal_graph(G, O):
    sc = S.small_grid(seed=S.BASE_SEED + 77)
    g, o = _pair(G, O, sc)
    p = G.setup(sc)
    p.set_outputs(ALL, 60, 3, 16)
    p.set_exec(G.SIM_EXEC_PERSISTENT, threads=256, blocks_per_sm=1)
    for k in range(4):
        g.step(250)
        p.step(250)
        o.step(250)
    compare_outputs(g, o, ALL, "graph")
    compare_outputs(p, o, ALL, "persistent")


def test_outputs_mid_run_clear(G, O):
    g, o = _pair(G, O, S.small_grid(), every=60, per=2, maxw=16)
    g.step(130)
    o.step(130)
    g.reset_outputs()
    o.reset_outputs()       # next sampling instant is step 180: window 1 holds one sample
    g.step(500)
    o.step(500)
    compare_outputs(g, o, ALL, "after clear")
    n = g.edge_samples()[2]
    assert n[0] == 0 and n[1] == 1 and n[2] == 2


def test_outputs_grid20_bitexact(G, O):
    g, o = _pair(G, O, S.grid(), every=120, per=6, maxw=5)
    for k in range(3):
        g.step(1200)
        o.step(1200)
        compare_outputs(g, o, ALL, f"grid20 step {1200 * (k + 1)}")
    compare(g, o, "grid20 end")


def test_outputs_metro_full_size_two_steps(G, O):
    sc = S.metro()
    off, links = S.random_walk_routes(sc, min_hops=10, max_hops=40)
    sc["routes"] = dict(offsets=off, links=links)
    sc["init_state"] = S.saturate(sc, off, links)
    g, o = _pair(G, O, sc, every=1, per=2, maxw=1)
    g.step(2)
    o.step(2)
    compare(g, o, "metro", check_occ=False)
    compare_outputs(g, o, ALL, "metro")
    assert g.edge_samples()[2][0] == 2


def test_outputs_batched_handle(G, O):
    scs = [S.small_grid(n=n, n_trips=150 * n, steps=700, seed=1100 + k, window_steps=400)
           for k, n in enumerate((5, 7, 6))]
    b = G.Sim.batch(scs)
    b.route()
    b.set_outputs(ALL, 50, 2, 8)
    oracles = []
    for sc in scs:
        o = O.OracleSim(sc)
        o.route()
        o.set_outputs(ALL, 50, 2, 8)
        oracles.append(o)
    b.step(700)
    for o in oracles:
        o.step(700)
    fb, cb = b.emissions()
    sb, nb = b.link_times()
    ub, vb, kb = b.edge_samples()
    t0 = l0 = 0
    for o, sc in zip(oracles, scs):
        nt, nl = sc["demand"]["n_trips"], sc["network"]["n_links"]
        fo, co = o.emissions()
        assert _same_bits(fb[t0:t0 + nt], fo) and _same_bits(cb[t0:t0 + nt], co)
        so, no = o.link_times()
        assert np.array_equal(sb[l0:l0 + nl], so) and np.array_equal(nb[l0:l0 + nl], no)
        uo, vo, ko = o.edge_samples()
        assert np.array_equal(kb, ko)
        assert _same_bits(ub[:, l0:l0 + nl], uo) and _same_bits(vb[:, l0:l0 + nl], vo)
        t0 += nt
        l0 += nl


# ---------------------------------------------------------------- reroute and equilibrium
def test_reroute_parity_small_metro(G, O):
    sc = S.small_metro()
    g, o = setup_pair(sc, G.Sim, O.OracleSim)
    rng = np.random.default_rng(11)
    for rnd, frac in ((1, 65536), (2, 32768), (3, 16384), (4, 0)):
        cost = rng.integers(10, 900, sc["network"]["n_links"]).astype(np.int32)
        g.reroute(cost, frac, rnd)
        o.reroute(cost, frac, rnd)
        for a, b in zip(g.routes(), o.routes()):
            assert np.array_equal(a, b), f"round {rnd}: routes differ"
    g.step(400)
    o.step(400)
    compare(g, o, "after reroutes")


def test_equilibrium_parity_small_grid(G, O):
    sc = S.small_grid(n_trips=900, window_steps=500)
    sc["params"]["cost_mode"] = 1
    g = G.Sim(sc)
    o = O.OracleSim(sc)
    g.set_outputs(2)
    o.set_outputs(2)
    cg, gg = g.equilibrium(SCHEDULE, 800)
    co, go = o.equilibrium(SCHEDULE, 800)
    assert np.array_equal(cg, co)
    assert _same_bits(gg, go), f"gaps {gg} vs {go}"
    for a, b in zip(g.routes(), o.routes()):
        assert np.array_equal(a, b)
    compare(g, o, "equilibrium end")
    assert gg[0] > 0


def test_equilibrium_parity_small_metro(G, O):
    sc = S.small_metro(n_trips=6000)
    sc["params"]["cost_mode"] = 1
    g = G.Sim(sc)
    o = O.OracleSim(sc)
    g.set_outputs(3)
    o.set_outputs(3)
    cg, gg = g.equilibrium(SCHEDULE, 1200)
    co, go = o.equilibrium(SCHEDULE, 1200)
    assert np.array_equal(cg, co)
    assert _same_bits(gg, go), f"gaps {gg} vs {go}"
    compare(g, o, "metro equilibrium end")
    compare_outputs(g, o, 3, "metro equilibrium end")


def test_output_error_codes(G):
    sc = S.small_grid()
    g = G.setup(sc)
    for call in (g.emissions, g.link_times, g.edge_samples):
        with pytest.raises(G.SimError) as e:
            call()
        assert e.value.code == G.SIM_ESTATE
    with pytest.raises(G.SimError) as e:
        g.measured_costs(np.ones(g.n_links, np.int32))
    assert e.value.code == G.SIM_ESTATE
    with pytest.raises(G.SimError) as e:
        g.set_outputs(8)
    assert e.value.code == G.SIM_EINVAL
    with pytest.raises(G.SimError) as e:
        g.set_outputs(4, 0, 6, 1)
    assert e.value.code == G.SIM_EINVAL
    with pytest.raises(G.SimError) as e:
        g.reroute(np.ones(g.n_links, np.int32), 65537, 1)
    assert e.value.code == G.SIM_EINVAL
    g.set_outputs(ALL, 10, 2, 3)         # windows cover steps 0 .. 59
    g.step(60)
    with pytest.raises(G.SimError) as e:
        g.step(1)
    assert e.value.code == G.SIM_EINVAL
    target = np.zeros((1, g.n_trips))
    with pytest.raises(G.SimError) as e:
        g.adjoint(20, 20, target, 1)
    assert e.value.code == G.SIM_ESTATE
    g.set_outputs(0)
    g.write_state(g.state())
    g.adjoint(20, 20, target, 1)         # outputs off: the adjoint runs
    g.set_outputs(1)
    with pytest.raises(G.SimError) as e:
        g.measured_costs(np.zeros(g.n_links, np.int32))
    assert e.value.code == G.SIM_ESTATE
